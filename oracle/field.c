/*
 * Boost-invariant classical Yang-Mills leapfrog on the transverse lattice
 * (test infrastructure; see oracle.h).
 *
 * Sec. 1 ("Glasma") of the paper: boost-invariant Glasma fields A(tau, x) in
 * Milne coordinates, evolved on the lattice in terms of gauge links and
 * plaquettes.  The lattice equations are those of the Hamiltonian (lattice
 * units, g absorbed):
 *   H(tau) = sum_x [ (1/tau) sum_i Tr E_i^2 + tau Tr pi^2 ] + V(tau),
 *   V(tau) = tau sum_x 2 (3 - Re Tr P(x))
 *          + (1/tau) sum_{x,i} Tr[(U_i(x) phi(x+i) U_i(x)^dag - phi(x))^2],
 *   P(x) = U_x(x) U_y(x+x) U_x(x+y)^dag U_y(x)^dag,  phi = A_eta, pi = dphi/dtau / tau,
 * with dU_i/dtau = i (E_i / tau) U_i and dphi/dtau = tau pi.  The kick is
 * E_i <- E_i - dtau grad_{U_i} V and pi <- pi - dtau dV/dphi, where
 * grad^a f(U) = d/de f(exp(i e t^a) U) at e = 0.  Worked out:
 *   dE_x/dtau = tau [ -ImTL P(x) + U_y(x-y)^dag ImTL P(x-y) U_y(x-y) ]
 *               - (1/tau) i [phi(x), U_x(x) phi(x+x) U_x(x)^dag]
 *   dE_y/dtau = tau [ +ImTL P(x) - U_x(x-x)^dag ImTL P(x-x) U_x(x-x) ]
 *               - (1/tau) i [phi(x), U_y(x) phi(x+y) U_y(x)^dag]
 *   dpi/dtau  = (1/tau) sum_i [ U_i(x) phi(x+i) U_i(x)^dag
 *               + U_i(x-i)^dag phi(x-i) U_i(x-i) - 2 phi(x) ]
 * with ImTL M = [(M - M^dag)/(2i)]_traceless.  One step (kick at tau_n, then
 * drift with tau_{n+1/2}):
 *   E_{n+1/2} = E_{n-1/2} + dtau F_E(tau_n),   pi likewise,
 *   U_{n+1}   = exp(i dtau E_{n+1/2} / tau_{n+1/2}) U_n,
 *   phi_{n+1} = phi_n + dtau tau_{n+1/2} pi_{n+1/2}.
 * expanding = 0 replaces every tau and 1/tau above by 1 (static box).
 *
 * Pins (tests/test_oracle_field.py): the force equals minus the numerical
 * group derivative of o_potential (4x4 brute force), gauge covariance of a
 * step, exact Gauss-law preservation, energy conservation (static box) with
 * O(dtau^2) oscillation, the Bjorken balance d(tau eps)/dtau = -P_L (expanding),
 * the abelian plane-wave dispersion, unitarity.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

static inline int site(int n, int x, int y) {
    x = (x % n + n) % n;
    y = (y % n + n) % n;
    return x + n * y;
}

static void plaquette(int n, const cplx *U, int x, int y, cplx P[9]) {
    const cplx *ux = U + 18 * site(n, x, y) + 0;
    const cplx *uy = U + 18 * site(n, x, y) + 9;
    const cplx *uyr = U + 18 * site(n, x + 1, y) + 9;
    const cplx *uxu = U + 18 * site(n, x, y + 1) + 0;
    cplx t[9];
    o_mul(ux, uyr, t);
    o_mul_dn(t, uxu, t);
    o_mul_dn(t, uy, P);
}

double o_potential(int n, double tau, int expanding, const cplx *U, const double *phi) {
    double tb = expanding ? tau : 1.0, tp = expanding ? 1.0 / tau : 1.0;
    double vb = 0, vp = 0;
    for (int y = 0; y < n; y++)
        for (int x = 0; x < n; x++) {
            cplx P[9];
            plaquette(n, U, x, y, P);
            vb += 2.0 * (3.0 - creal(P[0] + P[4] + P[8]));
            int s = site(n, x, y);
            for (int d = 0; d < 2; d++) {
                int sp = (d == 0) ? site(n, x + 1, y) : site(n, x, y + 1);
                double psi[8];
                o_conj_by(U + 18 * s + 9 * d, phi + 8 * sp, psi);
                /* Tr X^2 = (1/2) X^a X^a for X = psi - phi */
                for (int a = 0; a < 8; a++) {
                    double dd = psi[a] - phi[8 * s + a];
                    vp += 0.5 * dd * dd;
                }
            }
        }
    return tb * vb + tp * vp;
}

void o_force(int n, double tau, int expanding, const cplx *U, const double *phi, double *fE,
             double *fpi) {
    double tb = expanding ? tau : 1.0, tp = expanding ? 1.0 / tau : 1.0;
    size_t ns = (size_t)n * n;
    double *F = (double *)malloc(sizeof(double) * 8 * ns);
#pragma omp parallel for
    for (int s = 0; s < (int)ns; s++) {
        cplx P[9];
        plaquette(n, U, s % n, s / n, P);
        o_im_tl(P, F + 8 * s);
    }
#pragma omp parallel for
    for (int s = 0; s < (int)ns; s++) {
        int x = s % n, y = s / n;
        int sxm = site(n, x - 1, y), sym = site(n, x, y - 1);
        int sxp = site(n, x + 1, y), syp = site(n, x, y + 1);
        double tr[8], psi[8], cm[8], chi[8];
        /* E_x */
        o_transport(U + 18 * sym + 9, F + 8 * sym, tr);
        o_conj_by(U + 18 * s + 0, phi + 8 * sxp, psi);
        o_icomm(phi + 8 * s, psi, cm);
        for (int a = 0; a < 8; a++) fE[16 * s + a] = tb * (-F[8 * s + a] + tr[a]) - tp * cm[a];
        double lap[8];
        for (int a = 0; a < 8; a++) lap[a] = psi[a] - 2.0 * phi[8 * s + a];
        o_transport(U + 18 * sxm + 0, phi + 8 * sxm, chi);
        for (int a = 0; a < 8; a++) lap[a] += chi[a];
        /* E_y */
        o_transport(U + 18 * sxm + 0, F + 8 * sxm, tr);
        o_conj_by(U + 18 * s + 9, phi + 8 * syp, psi);
        o_icomm(phi + 8 * s, psi, cm);
        for (int a = 0; a < 8; a++) fE[16 * s + 8 + a] = tb * (F[8 * s + a] - tr[a]) - tp * cm[a];
        for (int a = 0; a < 8; a++) lap[a] += psi[a] - 2.0 * phi[8 * s + a];
        o_transport(U + 18 * sym + 9, phi + 8 * sym, chi);
        for (int a = 0; a < 8; a++) lap[a] += chi[a];
        for (int a = 0; a < 8; a++) fpi[8 * s + a] = tp * lap[a];
    }
    free(F);
}

void o_field_step(int n, int expanding, double dtau, int step, const cplx *U, const double *E,
                  const double *phi, const double *pi, cplx *U2, double *E2, double *phi2,
                  double *pi2) {
    size_t ns = (size_t)n * n;
    double tau_n = step * dtau, tau_h = (step + 0.5) * dtau;
    double *fE = (double *)malloc(sizeof(double) * 16 * ns);
    double *fpi = (double *)malloc(sizeof(double) * 8 * ns);
    o_force(n, tau_n, expanding, U, phi, fE, fpi);
    double ue = expanding ? dtau / tau_h : dtau;  /* coefficient of E in the link drift */
    double pe = expanding ? dtau * tau_h : dtau;  /* coefficient of pi in the phi drift */
#pragma omp parallel for
    for (int s = 0; s < (int)ns; s++) {
        for (int k = 0; k < 16; k++) E2[16 * s + k] = E[16 * s + k] + dtau * fE[16 * s + k];
        for (int a = 0; a < 8; a++) pi2[8 * s + a] = pi[8 * s + a] + dtau * fpi[8 * s + a];
        for (int d = 0; d < 2; d++) {
            double x[8];
            cplx W[9];
            for (int a = 0; a < 8; a++) x[a] = ue * E2[16 * s + 8 * d + a];
            o_exp_i(x, W);
            o_mul(W, U + 18 * s + 9 * d, U2 + 18 * s + 9 * d);
        }
        for (int a = 0; a < 8; a++) phi2[8 * s + a] = phi[8 * s + a] + pe * pi2[8 * s + a];
    }
    free(fE);
    free(fpi);
}

void o_reunitarize_all(int n, cplx *U) {
    for (int l = 0; l < 2 * n * n; l++) o_reunitarize(U + 9 * l);
}

void o_gauss(int n, const cplx *U, const double *E, const double *phi, const double *pi,
             double *G) {
    for (int y = 0; y < n; y++)
        for (int x = 0; x < n; x++) {
            int s = site(n, x, y);
            double g[8], tr[8], cm[8];
            for (int a = 0; a < 8; a++) g[a] = E[16 * s + a] + E[16 * s + 8 + a];
            int sxm = site(n, x - 1, y), sym = site(n, x, y - 1);
            o_transport(U + 18 * sxm + 0, E + 16 * sxm + 0, tr);
            for (int a = 0; a < 8; a++) g[a] -= tr[a];
            o_transport(U + 18 * sym + 9, E + 16 * sym + 8, tr);
            for (int a = 0; a < 8; a++) g[a] -= tr[a];
            o_icomm(phi + 8 * s, pi + 8 * s, cm);
            for (int a = 0; a < 8; a++) G[8 * s + a] = g[a] + cm[a];
        }
}

double o_gauss_rel(int n, const cplx *U, const double *E, const double *phi, const double *pi) {
    /* ||G|| relative to the scale of its terms: sum_x [2 sum_i |E_i(x)|^2 + |phi(x)|^2 |pi(x)|^2]
       (the transported E has the norm of E; |[phi, pi]| <= |phi| |pi| up to a constant) */
    size_t ns = (size_t)n * n;
    double *G = (double *)malloc(sizeof(double) * 8 * ns);
    o_gauss(n, U, E, phi, pi, G);
    double num = 0, den = 0;
    for (size_t s = 0; s < ns; s++) {
        double p2 = 0, q2 = 0;
        for (int a = 0; a < 8; a++) {
            num += G[8 * s + a] * G[8 * s + a];
            den += 2.0 * (E[16 * s + a] * E[16 * s + a] + E[16 * s + 8 + a] * E[16 * s + 8 + a]);
            p2 += phi[8 * s + a] * phi[8 * s + a];
            q2 += pi[8 * s + a] * pi[8 * s + a];
        }
        den += p2 * q2;
    }
    free(G);
    return den > 0 ? sqrt(num / den) : sqrt(num);
}

void o_energy(int n, double tau, int expanding, const cplx *U, const double *E,
              const double *phi, const double *pi, double out[4]) {
    double te = expanding ? tau : 1.0;
    double eet = 0, ebt = 0, eel = 0, ebl = 0;
    for (int y = 0; y < n; y++)
        for (int x = 0; x < n; x++) {
            int s = site(n, x, y);
            for (int a = 0; a < 16; a++) eet += 0.5 * E[16 * s + a] * E[16 * s + a];
            for (int a = 0; a < 8; a++) eel += 0.5 * pi[8 * s + a] * pi[8 * s + a];
            cplx P[9];
            plaquette(n, U, x, y, P);
            ebl += 2.0 * (3.0 - creal(P[0] + P[4] + P[8]));
            for (int d = 0; d < 2; d++) {
                int sp = (d == 0) ? site(n, x + 1, y) : site(n, x, y + 1);
                double psi[8];
                o_conj_by(U + 18 * s + 9 * d, phi + 8 * sp, psi);
                for (int a = 0; a < 8; a++) {
                    double dd = psi[a] - phi[8 * s + a];
                    ebt += 0.5 * dd * dd;
                }
            }
        }
    double ns = (double)n * n;
    out[0] = eet / (te * te) / ns;  /* eps_E,T */
    out[1] = ebt / (te * te) / ns;  /* eps_B,T */
    out[2] = eel / ns;              /* eps_E,L */
    out[3] = ebl / ns;              /* eps_B,L */
}

double o_unitarity_all(int n, const cplx *U) {
    double m = 0;
    for (int l = 0; l < 2 * n * n; l++) {
        double v = o_unitarity_dev(U + 9 * l);
        if (v > m) m = v;
    }
    return m;
}
