/*
 * MV-model initial conditions for the boost-invariant Glasma (test infrastructure).
 *
 * Sec. 1 ("Glasma", Eq. 1) of the paper: the color currents of the two nuclei
 * carry random charges rho^a(x) with <rho rho> ~ Qs^2 (McLerran-Venugopalan
 * model); the Glasma fields after the collision are solved on the transverse
 * lattice in terms of gauge links.  The paper defers the lattice formulas to its
 * companion paper, so the following standard readings are used:
 *   - rho^a_{A,n}(x) ~ N(0, (g^2 mu a)^2 / Ns), independent per nucleus A,
 *     longitudinal sheet n, site and color;
 *   - Lambda = (-lattice Laplacian + m^2)^-1 rho by FFT, lattice momentum
 *     k~^2 = sum_i 4 sin^2(pi n_i / N), zero mode set to 0;
 *   - V_A(x) = exp(-i Lambda_{A,Ns}) ... exp(-i Lambda_{A,1}) (sheet 1 rightmost);
 *   - pure-gauge nucleus links U^(A)_i(x) = V_A(x) V_A(x+i)^dagger;
 *   - tau = 0+ links: U_i(x) in SU(3) solving
 *       Im Tr[t^a (U^(1) + U^(2)) (1 + U^dagger)] = 0,  a = 1..8,
 *     by Newton's method in the chart U <- exp(i delta^b t^b) U, analytic Jacobian
 *     J_ab = -Re Tr[t^a (U^(1)+U^(2)) U^dagger t^b], step halving while the
 *     residual norm does not decrease, stop at ||r||_2 <= tol; start from
 *     U^(1) U^(2) (exact when the two links commute), restart once from 1 if
 *     the first attempt fails within max_iter iterations;
 *   - initial longitudinal field (E_i = phi = 0 at tau = 0):
 *       pi(x) = -(i/4) sum_i { [(U_i(x)-1)(U2_i(x)^dag - U1_i(x)^dag) - h.c.]
 *                + [(U_i(x-i)^dag - 1)(U2_i(x-i) - U1_i(x-i)) - h.c.] },
 *     which reduces to -i sum_i [A1_i, A2_i] at weak field;
 *   - first half step: E(tau_1/2) = 0, pi(tau_1/2) = pi(0), then one drift to
 *     tau_1 = dtau (U unchanged, phi = dtau * tau_1/2 * pi).
 *
 * Pins: tests/test_oracle_ic.py (Poisson solution satisfies the lattice
 * operator equation; abelian case U = U1 U2; residual and finite-difference
 * Jacobian; weak-field limit of pi(0); Gaussian moments of the charges).
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

void o_mv_charges(int n, int n_sheets, double g2mua, uint64_t seed, int nucleus,
                  int sheet, double *rho) {
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    double sigma = g2mua / sqrt((double)n_sheets);
    for (int s = 0; s < n * n; s++)
        for (int k = 0; k < 2; k++) {
            uint32_t ctr[4] = {(uint32_t)s, (uint32_t)(nucleus * n_sheets + sheet), (uint32_t)k, 1u};
            uint32_t r[4];
            o_philox4x32_10(ctr, key, r);
            double g0, g1, g2, g3;
            o_box_muller(r[0], r[1], &g0, &g1);
            o_box_muller(r[2], r[3], &g2, &g3);
            rho[8 * s + 4 * k + 0] = sigma * g0;
            rho[8 * s + 4 * k + 1] = sigma * g1;
            rho[8 * s + 4 * k + 2] = sigma * g2;
            rho[8 * s + 4 * k + 3] = sigma * g3;
        }
}

int o_poisson(int n, double m2, const double *rho, double *lam) {
    cplx *buf = (cplx *)malloc(sizeof(cplx) * n * n);
    if (!buf) return -1;
    for (int a = 0; a < 8; a++) {
        for (int s = 0; s < n * n; s++) buf[s] = rho[8 * s + a];
        o_fft2(n, buf, -1);
        for (int ky = 0; ky < n; ky++)
            for (int kx = 0; kx < n; kx++) {
                int s = kx + n * ky;
                if (kx == 0 && ky == 0) { buf[s] = 0; continue; }
                double sx = sin(M_PI * kx / n), sy = sin(M_PI * ky / n);
                double k2 = 4.0 * sx * sx + 4.0 * sy * sy;
                buf[s] /= (k2 + m2);
            }
        o_fft2(n, buf, +1);
        for (int s = 0; s < n * n; s++) lam[8 * s + a] = creal(buf[s]) / ((double)n * n);
    }
    free(buf);
    return 0;
}

int o_wilson_line(int n, int n_sheets, double g2mua, double m_ir_a, uint64_t seed,
                  int nucleus, cplx *V) {
    double *rho = (double *)malloc(sizeof(double) * 8 * n * n);
    double *lam = (double *)malloc(sizeof(double) * 8 * n * n);
    if (!rho || !lam) { free(rho); free(lam); return -1; }
    for (int s = 0; s < n * n; s++)
        for (int k = 0; k < 9; k++) V[9 * s + k] = (k % 4 == 0) ? 1.0 : 0.0;
    for (int sh = 0; sh < n_sheets; sh++) {
        o_mv_charges(n, n_sheets, g2mua, seed, nucleus, sh, rho);
        if (o_poisson(n, m_ir_a * m_ir_a, rho, lam)) { free(rho); free(lam); return -1; }
        for (int s = 0; s < n * n; s++) {
            double x[8];
            cplx W[9];
            for (int a = 0; a < 8; a++) x[a] = -lam[8 * s + a];
            o_exp_i(x, W);
            o_mul(W, V + 9 * s, V + 9 * s);
        }
    }
    free(rho);
    free(lam);
    return 0;
}

void o_pure_gauge_links(int n, const cplx *V, cplx *UA) {
    for (int y = 0; y < n; y++)
        for (int x = 0; x < n; x++) {
            int s = site(n, x, y);
            o_mul_dn(V + 9 * s, V + 9 * site(n, x + 1, y), UA + 18 * s + 0);
            o_mul_dn(V + 9 * s, V + 9 * site(n, x, y + 1), UA + 18 * s + 9);
        }
}

void o_ic_residual(const cplx U1[9], const cplx U2[9], const cplx U[9], double r[8]) {
    cplx S[9], M[9], Ud[9], T[9];
    for (int k = 0; k < 9; k++) S[k] = U1[k] + U2[k];
    o_dag(U, Ud);
    for (int k = 0; k < 9; k++) M[k] = Ud[k] + ((k % 4 == 0) ? 1.0 : 0.0);
    o_mul(S, M, M);
    for (int a = 0; a < 8; a++) {
        o_generator(a, T);
        cplx tr = 0;
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) tr += T[3 * i + j] * M[3 * j + i];
        r[a] = cimag(tr);
    }
}

void o_ic_jacobian(const cplx U1[9], const cplx U2[9], const cplx U[9], double J[64]) {
    cplx S[9], SUd[9], Ta[9], Tb[9], A[9], B[9];
    for (int k = 0; k < 9; k++) S[k] = U1[k] + U2[k];
    o_mul_dn(S, U, SUd);
    for (int a = 0; a < 8; a++) {
        o_generator(a, Ta);
        o_mul(Ta, SUd, A);
        for (int b = 0; b < 8; b++) {
            o_generator(b, Tb);
            o_mul(A, Tb, B);
            J[8 * a + b] = -creal(B[0] + B[4] + B[8]);
        }
    }
}

/* Gaussian elimination with partial pivoting, 8x8; returns 0 on success */
static int solve8(double A[64], double b[8], double x[8]) {
    double M[8][9];
    for (int i = 0; i < 8; i++) {
        for (int j = 0; j < 8; j++) M[i][j] = A[8 * i + j];
        M[i][8] = b[i];
    }
    for (int c = 0; c < 8; c++) {
        int p = c;
        for (int i = c + 1; i < 8; i++)
            if (fabs(M[i][c]) > fabs(M[p][c])) p = i;
        if (fabs(M[p][c]) < 1e-300) return -1;
        if (p != c)
            for (int j = 0; j < 9; j++) { double t = M[c][j]; M[c][j] = M[p][j]; M[p][j] = t; }
        for (int i = c + 1; i < 8; i++) {
            double f = M[i][c] / M[c][c];
            for (int j = c; j < 9; j++) M[i][j] -= f * M[c][j];
        }
    }
    for (int i = 7; i >= 0; i--) {
        double s = M[i][8];
        for (int j = i + 1; j < 8; j++) s -= M[i][j] * x[j];
        x[i] = s / M[i][i];
    }
    return 0;
}

static double norm8(const double r[8]) {
    double s = 0;
    for (int a = 0; a < 8; a++) s += r[a] * r[a];
    return sqrt(s);
}

int o_ic_solve_link(const cplx U1[9], const cplx U2[9], cplx U[9], double tol,
                    int max_iter, double *res_out) {
    double r[8], J[64], d[8];
    o_ic_residual(U1, U2, U, r);
    double rn = norm8(r);
    int it = 0;
    while (rn > tol && it < max_iter) {
        o_ic_jacobian(U1, U2, U, J);
        double mr[8];
        for (int a = 0; a < 8; a++) mr[a] = -r[a];
        if (solve8(J, mr, d)) break;
        /* step halving: accept the first step length that lowers ||r|| */
        double lam = 1.0;
        cplx Un[9];
        double rnew[8], rnn = 0;
        for (int h = 0; h < 12; h++) {
            double dx[8];
            cplx W[9];
            for (int a = 0; a < 8; a++) dx[a] = lam * d[a];
            o_exp_i(dx, W);
            o_mul(W, U, Un);
            o_ic_residual(U1, U2, Un, rnew);
            rnn = norm8(rnew);
            if (rnn < rn) break;
            lam *= 0.5;
        }
        it++;
        if (!(rnn < rn)) { rn = rnn; memcpy(U, Un, sizeof(Un)); memcpy(r, rnew, sizeof(rnew)); break; }
        memcpy(U, Un, sizeof(Un));
        memcpy(r, rnew, sizeof(rnew));
        rn = rnn;
    }
    if (res_out) *res_out = rn;
    return rn <= tol ? it : -1;
}

int o_ic_solve(int n, const cplx *U1, const cplx *U2, const cplx *U_start, double tol,
               int max_iter, cplx *U, int32_t *iters, double *res) {
    int fails = 0;
#pragma omp parallel for reduction(+ : fails) schedule(dynamic, 64)
    for (int l = 0; l < 2 * n * n; l++) {
        cplx *u = U + 9 * l;
        /* start: the caller's guess, else U1 U2 (the exact root when the two
           nuclei's links commute); if Newton stalls, restart once from 1 */
        if (U_start)
            memcpy(u, U_start + 9 * l, sizeof(cplx) * 9);
        else
            o_mul(U1 + 9 * l, U2 + 9 * l, u);
        double rr;
        int it = o_ic_solve_link(U1 + 9 * l, U2 + 9 * l, u, tol, max_iter, &rr);
        if (it < 0) {
            int spent = max_iter;
            for (int k = 0; k < 9; k++) u[k] = (k % 4 == 0) ? 1.0 : 0.0;
            it = o_ic_solve_link(U1 + 9 * l, U2 + 9 * l, u, tol, max_iter, &rr);
            if (it >= 0) it += spent;
        }
        if (iters) iters[l] = it;
        if (res) res[l] = rr;
        if (it < 0) fails++;
    }
    return fails;
}

void o_pi0(int n, const cplx *U, const cplx *U1, const cplx *U2, double *pi) {
    for (int y = 0; y < n; y++)
        for (int x = 0; x < n; x++) {
            int s = site(n, x, y);
            cplx M[9];
            for (int k = 0; k < 9; k++) M[k] = 0;
            for (int d = 0; d < 2; d++) {
                int sm = (d == 0) ? site(n, x - 1, y) : site(n, x, y - 1);
                const cplx *u = U + 18 * s + 9 * d, *u1 = U1 + 18 * s + 9 * d,
                           *u2 = U2 + 18 * s + 9 * d;
                const cplx *um = U + 18 * sm + 9 * d, *u1m = U1 + 18 * sm + 9 * d,
                           *u2m = U2 + 18 * sm + 9 * d;
                cplx A[9], B[9], C[9], Cd[9];
                /* (U(x) - 1)(U2(x)^dag - U1(x)^dag) */
                for (int k = 0; k < 9; k++) A[k] = u[k] - ((k % 4 == 0) ? 1.0 : 0.0);
                for (int i = 0; i < 3; i++)
                    for (int j = 0; j < 3; j++) B[3 * i + j] = conj(u2[3 * j + i]) - conj(u1[3 * j + i]);
                o_mul(A, B, C);
                o_dag(C, Cd);
                for (int k = 0; k < 9; k++) M[k] += C[k] - Cd[k];
                /* (U(x-i)^dag - 1)(U2(x-i) - U1(x-i)) */
                for (int i = 0; i < 3; i++)
                    for (int j = 0; j < 3; j++)
                        A[3 * i + j] = conj(um[3 * j + i]) - ((i == j) ? 1.0 : 0.0);
                for (int k = 0; k < 9; k++) B[k] = u2m[k] - u1m[k];
                o_mul(A, B, C);
                o_dag(C, Cd);
                for (int k = 0; k < 9; k++) M[k] += C[k] - Cd[k];
            }
            for (int k = 0; k < 9; k++) M[k] *= -0.25 * I;
            o_mat_to_alg(M, pi + 8 * s);
        }
}

int o_glasma_init(int n, int n_sheets, double g2mua, double m_ir_a, uint64_t seed,
                  double dtau, double tol, int max_iter, cplx *U, double *E, double *phi,
                  double *pi, int32_t *iters) {
    size_t ns = (size_t)n * n;
    cplx *V1 = (cplx *)malloc(sizeof(cplx) * 9 * ns), *V2 = (cplx *)malloc(sizeof(cplx) * 9 * ns);
    cplx *U1 = (cplx *)malloc(sizeof(cplx) * 18 * ns), *U2 = (cplx *)malloc(sizeof(cplx) * 18 * ns);
    int rc = 0;
    if (!V1 || !V2 || !U1 || !U2) { rc = -1; goto done; }
    if (o_wilson_line(n, n_sheets, g2mua, m_ir_a, seed, 0, V1) ||
        o_wilson_line(n, n_sheets, g2mua, m_ir_a, seed, 1, V2)) { rc = -1; goto done; }
    o_pure_gauge_links(n, V1, U1);
    o_pure_gauge_links(n, V2, U2);
    rc = o_ic_solve(n, U1, U2, NULL, tol, max_iter, U, iters, NULL);
    o_pi0(n, U, U1, U2, pi);
    /* state at step 1: U_1 = U_0, E_1/2 = 0, pi_1/2 = pi(0), phi_1 = dtau * (dtau/2) * pi */
    memset(E, 0, sizeof(double) * 16 * ns);
    for (size_t k = 0; k < 8 * ns; k++) phi[k] = dtau * (0.5 * dtau) * pi[k];
done:
    free(V1); free(V2); free(U1); free(U2);
    return rc;
}
