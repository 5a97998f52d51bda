/*
 * FP64 reference of the lattice-correlator estimators of the momentum broadening
 * (Sec. 2, "Lattice correlators", Eqs. 4 and 5 of arXiv:2307.07999; test
 * infrastructure, see oracle.h).
 *
 * Static quarks (m -> infinity, Eq. 4): at every site x the running integral
 *   I_i(x, tau) = sum over steps of dtau * E_i(x, tau_n),
 * with E_i the site-centred fields of the particle push (o_gather: E_x, E_y averaged
 * over the two links touching the site and over tau_{n +- 1/2}, divided by tau; E_z the
 * time-centred pi), so that <dp_i^2> = < Tr I_i^2 > = < (1/2) sum_a (I_i^a)^2 >, the
 * average over x standing for the average over quark positions and colour charges
 * (<Q^a Q^b> = delta^ab / 2).
 *
 * Lightlike jets along +x (p_x -> infinity, Eq. 5): from every start site x0 a path
 * moving one lattice unit of x per lattice unit of tau, starting at offset ox0 in its
 * cell; after m steps it sits in cell x0 + k(m), k(m) = floor(ox0 + m dtau).  The force
 * combinations F_x = E_x, F_y = E_y - B_z, F_z = E_z + B_y at the path's cell are
 * carried back to x0 by the path's Wilson line W = U_x(x0) U_x(x0+1) ... (one link per
 * cell crossed):  J_i(x0) += dtau * W F_i W^dag, and W <- W U_x(c) when the path leaves
 * cell c (links at tau_n).  <dp_i^2> = < (1/2) sum_a (J_i^a)^2 >.  This is what a
 * colour charge Q0 would collect while parallel transported along the path (the push
 * rotates Q <- U^dag Q U on crossing), averaged over Q0.
 *
 * Both start at the step where particles formed at the same time take their first
 * kick, and use the fields of that step exactly as o_push does.
 * Pins (tests/test_oracle_correlators.py): the closed form of a uniform Cartan E field;
 * the static limit of o_push (m -> infinity) and its lightlike limit (p_x -> infinity)
 * for every site's charge; gauge invariance of both estimators.
 */
#include <math.h>
#include <string.h>
#include "oracle.h"

static inline int wrap(int n, int v) { return ((v % n) + n) % n; }

void o_corr_step(int n, int expanding, double dtau, int step, const cplx *U, const double *Eo,
                 const double *En, const double *phi, const double *pio, const double *pin,
                 double *Istat, cplx *W, double *J, int k_now, int k_next, double out[6]) {
    const double tau_n = step * dtau;
    double s_stat[3] = {0, 0, 0}, s_light[3] = {0, 0, 0};
#pragma omp parallel for reduction(+ : s_stat[:3], s_light[:3])
    for (int s = 0; s < n * n; s++) {
        const int x = s % n, y = s / n;
        double F[6][8];
        /* static: the site's own fields */
        o_gather(n, tau_n, expanding, U, Eo, En, phi, pio, pin, x, y, F);
        double *Is = Istat + 24 * s;
        for (int i = 0; i < 3; i++)
            for (int a = 0; a < 8; a++) Is[8 * i + a] += dtau * F[i][a];
        for (int i = 0; i < 3; i++) {
            double q = 0;
            for (int a = 0; a < 8; a++) q += Is[8 * i + a] * Is[8 * i + a];
            s_stat[i] += 0.5 * q;
        }
        /* lightlike: the path from x0 = (x, y) is in cell (x + k_now, y) */
        const int cx = wrap(n, x + k_now);
        o_gather(n, tau_n, expanding, U, Eo, En, phi, pio, pin, cx, y, F);
        double Fl[3][8];
        for (int a = 0; a < 8; a++) {
            Fl[0][a] = F[0][a];
            Fl[1][a] = F[1][a] - F[5][a];
            Fl[2][a] = F[2][a] + F[4][a];
        }
        cplx *w = W + 9 * s;
        double *Jl = J + 24 * s;
        for (int i = 0; i < 3; i++) {
            double t[8];
            o_conj_by(w, Fl[i], t); /* W F W^dag */
            double q = 0;
            for (int a = 0; a < 8; a++) {
                Jl[8 * i + a] += dtau * t[a];
                q += Jl[8 * i + a] * Jl[8 * i + a];
            }
            s_light[i] += 0.5 * q;
        }
        if (k_next > k_now) {
            cplx t[9];
            o_mul(w, U + 18 * (cx + n * y) + 0, t);
            memcpy(w, t, sizeof(t));
        }
    }
    for (int i = 0; i < 3; i++) {
        out[i] = s_stat[i] / (n * n);
        out[3 + i] = s_light[i] / (n * n);
    }
}
