/*
 * Colored particle-in-cell solution of Wong's equations (test infrastructure).
 *
 * Sec. 1 ("Probes in Glasma", Eq. 2) of the paper: dx^mu/dtau = p^mu/m,
 * Dp^mu/dtau = 2g Tr{Q F^{mu nu}} p_nu / m, and the color charge is rotated with
 * particle Wilson lines built from the lattice gauge links, Q -> U Q U^dag,
 * which conserves q2 = Q^a Q^a and q3 = d_abc Q^a Q^b Q^c.  Q0 and the Haar
 * rotation follow the same paragraph: Q0 in the Cartan subalgebra with the
 * given q2, q3, then Q(tau0) = U Q0 U^dag with Haar U; <Q^a Q^b> = delta/2 and
 * <Q^a Q^b Q^c> = d^abc/4 fix q2 = 4, q3 = 10/3.
 *
 * Milne-coordinate form (lattice units, coordinate time tau; p_eta^ = tau p^eta;
 * p^tau = sqrt(m^2 + px^2 + py^2 + p_eta^2)); 2Tr(Q F) = Q^a F^a:
 *   dpx/dtau    = Q.[Ex + (py Bz - peta By)/p^tau]
 *   dpy/dtau    = Q.[Ey + (peta Bx - px Bz)/p^tau]
 *   dpeta/dtau  = Q.[Ez + (px By - py Bx)/p^tau] - peta/tau
 *   dx/dtau = px/p^tau, dy/dtau = py/p^tau, deta/dtau = peta/(tau p^tau)
 * (the -peta/tau term is the Christoffel term of the Milne metric).  The
 * lightlike limit of Sec. 2 (Eq. 5: F_y = E_y - B_z, F_z = E_z + B_y at v_x = 1)
 * fixes the sign convention of the magnetic force.
 *
 * Site-centred fields at the particle's nearest-grid-point cell c at tau_n
 * (readings; the paper defers the discretisation to its companion paper):
 *   Ex = (1/2)[E^_x(c) + U_x(c-x)^dag E^_x(c-x) U_x(c-x)] / tau_n,
 *        E^ = (E_{n-1/2} + E_{n+1/2})/2;  Ey likewise;  Ez = (pi_{n-1/2}+pi_{n+1/2})/2;
 *   D_iphi = (1/2)[U_i(c) phi(c+i) U_i(c)^dag - U_i(c-i)^dag phi(c-i) U_i(c-i)],
 *   Bx = -D_yphi / tau_n,  By = +D_xphi / tau_n,
 *   Bz = -F_xy,  F_xy = (1/4) ImTL(sum of the four plaquettes at c, all
 *        counter-clockwise and based at c)  (clover).
 * One push from tau_n to tau_{n+1}: kick p with the pre-step p in the magnetic
 * term; drift x, y, eta with the new p (eta with tau_{n+1/2}); rotate Q by
 * exp(-i phi_n(c) deta) first, then across the x face (Q <- U_x(c)^dag Q U_x(c) on
 * +x, Q <- U_x(c-x) Q U_x(c-x)^dag on -x), then across the y face from the new
 * x cell.  Broadening terms dp_i^2 = p_i^2 - p_i(tau_form)^2 with the lab
 * p_z = p^tau sinh(eta) + p_eta^ cosh(eta) (Sec. 2, "Quantifying the effect").
 * expanding = 0: every tau factor -> 1, eta -> z, no Christoffel term.
 *
 * Pins (tests/test_oracle_particles.py): free streaming, pure-gauge color
 * transport, gauge invariance of p(tau), Casimir conservation, constant
 * Cartan E field, cyclotron motion in a uniform Cartan B field (first order
 * convergence), static and lightlike limits, Q ensemble moments.
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

static double dot8(const double a[8], const double b[8]) {
    double s = 0;
    for (int k = 0; k < 8; k++) s += a[k] * b[k];
    return s;
}

void o_casimirs(const double Q[8], double *q2, double *q3) {
    static double f[512], d[512];
    static int ready = 0;
    if (!ready) { o_structure_constants(f, d); ready = 1; }
    double s2 = 0, s3 = 0;
    for (int a = 0; a < 8; a++) {
        s2 += Q[a] * Q[a];
        for (int b = 0; b < 8; b++)
            for (int c = 0; c < 8; c++) s3 += d[64 * a + 8 * b + c] * Q[a] * Q[b] * Q[c];
    }
    *q2 = s2;
    *q3 = s3;
}

void o_q0_cartan(double q2, double q3, double Q0[8]) {
    /* q3 = (1/sqrt3)(3 q2 Q8 - 4 Q8^3), Q3 = sqrt(q2 - Q8^2): depressed cubic
       Q8^3 + p Q8 + q = 0 with p = -3 q2 / 4, q = sqrt3 q3 / 4; trigonometric roots,
       take the smallest positive one (all three are Weyl-equivalent). */
    double p = -0.75 * q2, q = sqrt(3.0) * q3 / 4.0;
    double m = 2.0 * sqrt(-p / 3.0);
    double arg = (3.0 * q / (2.0 * p)) * sqrt(-3.0 / p);
    if (arg > 1) arg = 1;
    if (arg < -1) arg = -1;
    double th = acos(arg) / 3.0;
    double best = 1e300;
    for (int k = 0; k < 3; k++) {
        double r = m * cos(th - 2.0 * M_PI * k / 3.0);
        if (r > 0 && r < best) best = r;
    }
    for (int a = 0; a < 8; a++) Q0[a] = 0;
    Q0[7] = best;
    Q0[2] = sqrt(fmax(q2 - best * best, 0.0));
}

void o_particles_init(int np, int n, double mass, int init_kind, double p_min, double p_max,
                      double q2, double q3, uint64_t seed, double *x, double *y, double *eta,
                      double *px, double *py, double *peta, double *Q) {
    (void)mass;
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    double Q0[8];
    o_q0_cartan(q2, q3, Q0);
    for (int j = 0; j < np; j++) {
        uint32_t ctr[4] = {(uint32_t)j, 0u, 0u, 2u}, r[4];
        o_philox4x32_10(ctr, key, r);
        x[j] = n * o_u01(r[0]);
        y[j] = n * o_u01(r[1]);
        double pm = p_min + (p_max - p_min) * o_u01(r[2]);
        double az = 2.0 * M_PI * o_u01(r[3]);
        if (init_kind == 0) {          /* |p_T| uniform, isotropic azimuth */
            px[j] = pm * cos(az);
            py[j] = pm * sin(az);
        } else {                       /* along +x, |p| uniform in [p_min, p_max] */
            px[j] = pm;
            py[j] = 0.0;
        }
        eta[j] = 0.0;
        peta[j] = 0.0;
        double g[20];
        for (int k = 1; k <= 5; k++) {
            uint32_t c2[4] = {(uint32_t)j, 0u, (uint32_t)k, 2u};
            o_philox4x32_10(c2, key, r);
            o_box_muller(r[0], r[1], &g[4 * (k - 1) + 0], &g[4 * (k - 1) + 1]);
            o_box_muller(r[2], r[3], &g[4 * (k - 1) + 2], &g[4 * (k - 1) + 3]);
        }
        cplx U[9];
        o_haar(g, U);
        o_conj_by(U, Q0, Q + 8 * j);
    }
}

void o_gather(int n, double tau, int expanding, const cplx *U, const double *Eo,
              const double *En, const double *phi, const double *pio, const double *pin,
              int cx, int cy, double F[6][8]) {
    double te = expanding ? tau : 1.0;
    int c = site(n, cx, cy);
    int cxm = site(n, cx - 1, cy), cym = site(n, cx, cy - 1);
    int cxp = site(n, cx + 1, cy), cyp = site(n, cx, cy + 1);
    double eb[8], ebm[8], tr[8];
    /* E_x, E_y : average of the two links touching c, time-centred */
    for (int d = 0; d < 2; d++) {
        int cm = d == 0 ? cxm : cym;
        for (int a = 0; a < 8; a++) {
            eb[a] = 0.5 * (Eo[16 * c + 8 * d + a] + En[16 * c + 8 * d + a]);
            ebm[a] = 0.5 * (Eo[16 * cm + 8 * d + a] + En[16 * cm + 8 * d + a]);
        }
        o_transport(U + 18 * cm + 9 * d, ebm, tr);
        for (int a = 0; a < 8; a++) F[d][a] = 0.5 * (eb[a] + tr[a]) / te;
    }
    for (int a = 0; a < 8; a++) F[2][a] = 0.5 * (pio[8 * c + a] + pin[8 * c + a]);
    /* covariant central differences of phi */
    double dphi[2][8];
    for (int d = 0; d < 2; d++) {
        int cp = d == 0 ? cxp : cyp, cm = d == 0 ? cxm : cym;
        double fw[8], bw[8];
        o_conj_by(U + 18 * c + 9 * d, phi + 8 * cp, fw);
        o_transport(U + 18 * cm + 9 * d, phi + 8 * cm, bw);
        for (int a = 0; a < 8; a++) dphi[d][a] = 0.5 * (fw[a] - bw[a]);
    }
    for (int a = 0; a < 8; a++) {
        F[3][a] = -dphi[1][a] / te;  /* B_x */
        F[4][a] = dphi[0][a] / te;   /* B_y */
    }
    /* clover F_xy at c */
    const cplx *ux_c = U + 18 * c, *uy_c = U + 18 * c + 9;
    const cplx *ux_xm = U + 18 * cxm, *uy_xm = U + 18 * cxm + 9;
    const cplx *ux_ym = U + 18 * cym, *uy_ym = U + 18 * cym + 9;
    const cplx *uy_xp = U + 18 * cxp + 9, *ux_yp = U + 18 * cyp;
    const cplx *ux_xmyp = U + 18 * site(n, cx - 1, cy + 1);
    const cplx *uy_xmym = U + 18 * site(n, cx - 1, cy - 1) + 9;
    const cplx *ux_xmym = U + 18 * site(n, cx - 1, cy - 1);
    const cplx *uy_xpym = U + 18 * site(n, cx + 1, cy - 1) + 9;
    cplx S[9], P[9], t[9], d[9];
    for (int k = 0; k < 9; k++) S[k] = 0;
    /* +x,+y: U_x(c) U_y(c+x) U_x(c+y)^dag U_y(c)^dag */
    o_mul(ux_c, uy_xp, t); o_mul_dn(t, ux_yp, t); o_mul_dn(t, uy_c, P);
    for (int k = 0; k < 9; k++) S[k] += P[k];
    /* +y,-x: U_y(c) U_x(c-x+y)^dag U_y(c-x)^dag U_x(c-x) */
    o_mul_dn(uy_c, ux_xmyp, t); o_mul_dn(t, uy_xm, t); o_mul(t, ux_xm, P);
    for (int k = 0; k < 9; k++) S[k] += P[k];
    /* -x,-y: U_x(c-x)^dag U_y(c-x-y)^dag U_x(c-x-y) U_y(c-y) */
    o_dag(ux_xm, d); o_mul_dn(d, uy_xmym, t); o_mul(t, ux_xmym, t); o_mul(t, uy_ym, P);
    for (int k = 0; k < 9; k++) S[k] += P[k];
    /* -y,+x: U_y(c-y)^dag U_x(c-y) U_y(c+x-y) U_x(c)^dag */
    o_dag(uy_ym, d); o_mul(d, ux_ym, t); o_mul(t, uy_xpym, t); o_mul_dn(t, ux_c, P);
    for (int k = 0; k < 9; k++) S[k] += P[k];
    double fxy[8];
    o_im_tl(S, fxy);
    for (int a = 0; a < 8; a++) F[5][a] = -0.25 * fxy[a];  /* B_z = -F_xy */
}

/* Cloud-in-cell gather (reading; the paper does not give the interpolation): the
 * site-centred fields of the four sites around the particle, c, c+x, c+y, c+x+y, each
 * parallel transported into the frame of c where Q lives (c+x by U_x(c), c+y by U_y(c),
 * c+x+y by U_y(c+x) and then U_x(c): x before y, as the colour crossings), weighted
 * bilinearly with the particle's offsets (ox, oy) in the cell. */
void o_gather_cic(int n, double tau, int expanding, const cplx *U, const double *Eo, const double *En,
                  const double *phi, const double *pio, const double *pin, int cx, int cy, double ox,
                  double oy, double F[6][8]) {
    const double w[4] = {(1 - ox) * (1 - oy), ox * (1 - oy), (1 - ox) * oy, ox * oy};
    const int sx[4] = {cx, cx + 1, cx, cx + 1}, sy[4] = {cy, cy, cy + 1, cy + 1};
    for (int i = 0; i < 6; i++)
        for (int a = 0; a < 8; a++) F[i][a] = 0.0;
    for (int k = 0; k < 4; k++) {
        double Fk[6][8];
        o_gather(n, tau, expanding, U, Eo, En, phi, pio, pin, sx[k], sy[k], Fk);
        for (int i = 0; i < 6; i++) {
            double t[8];
            if (k == 3) { /* c+x+y -> c+x -> c */
                o_conj_by(U + 18 * site(n, cx + 1, cy) + 9, Fk[i], t);
                o_conj_by(U + 18 * site(n, cx, cy) + 0, t, Fk[i]);
            } else if (k == 1) {
                o_conj_by(U + 18 * site(n, cx, cy) + 0, Fk[i], t);
                memcpy(Fk[i], t, sizeof(t));
            } else if (k == 2) {
                o_conj_by(U + 18 * site(n, cx, cy) + 9, Fk[i], t);
                memcpy(Fk[i], t, sizeof(t));
            }
            for (int a = 0; a < 8; a++) F[i][a] += w[k] * Fk[i][a];
        }
    }
}

double o_pz_lab(double mass, double px, double py, double peta, double eta) {
    double pt = sqrt(mass * mass + px * px + py * py + peta * peta);
    return pt * sinh(eta) + peta * cosh(eta);
}

void o_push(int np, int n, int expanding, double dtau, int step, double mass, const cplx *U,
            const double *Eo, const double *En, const double *phi, const double *pio,
            const double *pin, double *x, double *y, double *eta, double *px, double *py,
            double *peta, double *Q, const double *p0, double acc[4]) {
    o_push_int(np, n, expanding, dtau, step, mass, U, Eo, En, phi, pio, pin, x, y, eta, px, py, peta, Q,
               p0, acc, 0);
}

/* The momentum kick of one step with the charge-contracted fields qE, qB (both
 * integrators; the Christoffel term -p_eta^/tau acts only when expanding).
 *   explicit (0): p += dtau [qE + (p / p^tau) x qB] - dtau p_eta^/tau_n e_eta (first order)
 *   Boris (1):    p_eta^ *= tau_n / tau_{n+1/2} (exact decay over the first half step);
 *                 p- = p + dtau/2 qE;  rotation of p- about qB by the angle of
 *                 t = (dtau/2) qB / p^tau(p-):  p' = p- + p- x t,  p+ = p- + p' x 2t/(1 + t.t)
 *                 (|p+| = |p-| exactly);  p = p+ + dtau/2 qE;
 *                 p_eta^ *= tau_{n+1/2} / tau_{n+1}   (second order, Boris 1970) */
static void kick(int integrator, int expanding, double dtau, double tau_n, double mass, const double qE[3],
                 const double qB[3], double p[3]) {
    if (integrator == 0) {
        const double pt = sqrt(mass * mass + p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
        const double ipt = pt > 0 ? 1.0 / pt : 0.0;
        double f[3] = {qE[0] + (p[1] * qB[2] - p[2] * qB[1]) * ipt, qE[1] + (p[2] * qB[0] - p[0] * qB[2]) * ipt,
                       qE[2] + (p[0] * qB[1] - p[1] * qB[0]) * ipt};
        if (expanding) f[2] -= p[2] / tau_n;
        for (int i = 0; i < 3; i++) p[i] += dtau * f[i];
        return;
    }
    const double tau_h = tau_n + 0.5 * dtau, tau_1 = tau_n + dtau;
    if (expanding) p[2] *= tau_n / tau_h;
    for (int i = 0; i < 3; i++) p[i] += 0.5 * dtau * qE[i];
    const double g = sqrt(mass * mass + p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
    const double ig = g > 0 ? 1.0 / g : 0.0;
    const double t[3] = {0.5 * dtau * qB[0] * ig, 0.5 * dtau * qB[1] * ig, 0.5 * dtau * qB[2] * ig};
    const double pp[3] = {p[0] + (p[1] * t[2] - p[2] * t[1]), p[1] + (p[2] * t[0] - p[0] * t[2]),
                          p[2] + (p[0] * t[1] - p[1] * t[0])};
    const double sf = 2.0 / (1.0 + t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    p[0] += sf * (pp[1] * t[2] - pp[2] * t[1]);
    p[1] += sf * (pp[2] * t[0] - pp[0] * t[2]);
    p[2] += sf * (pp[0] * t[1] - pp[1] * t[0]);
    for (int i = 0; i < 3; i++) p[i] += 0.5 * dtau * qE[i];
    if (expanding) p[2] *= tau_h / tau_1;
}

void o_push_ext(int np, int n, int expanding, double dtau, int step, double mass, const cplx *U,
                const double *Eo, const double *En, const double *phi, const double *pio,
                const double *pin, double *x, double *y, double *eta, double *px, double *py,
                double *peta, double *Q, const double *p0, double acc[4], int integrator, int substeps,
                int interp);

void o_push_int(int np, int n, int expanding, double dtau, int step, double mass, const cplx *U,
                const double *Eo, const double *En, const double *phi, const double *pio,
                const double *pin, double *x, double *y, double *eta, double *px, double *py,
                double *peta, double *Q, const double *p0, double acc[4], int integrator) {
    o_push_ext(np, n, expanding, dtau, step, mass, U, Eo, En, phi, pio, pin, x, y, eta, px, py, peta, Q, p0, acc,
               integrator, 1, 0);
}

/* The push of one field step taken as `substeps` particle steps of h = dtau / substeps.
 * The fields stay those of the step (gathered at the particle's current cell in every
 * sub-step, E and D phi divided by tau_n); the sub-step k from tau_k = tau_n + k h kicks
 * with h at tau_k, drifts with h (eta with tau_k + h/2) and rotates the colour as one
 * step does.  The broadening terms are taken after the last sub-step. */
void o_push_sub(int np, int n, int expanding, double dtau, int step, double mass, const cplx *U,
                const double *Eo, const double *En, const double *phi, const double *pio,
                const double *pin, double *x, double *y, double *eta, double *px, double *py,
                double *peta, double *Q, const double *p0, double acc[4], int integrator, int substeps) {
    o_push_ext(np, n, expanding, dtau, step, mass, U, Eo, En, phi, pio, pin, x, y, eta, px, py, peta, Q, p0, acc,
               integrator, substeps, 0);
}

/* o_push_sub with the gather chosen by interp: 0 nearest grid point (the site at the
 * lower-left corner of the particle's cell), 1 cloud in cell (o_gather_cic). */
void o_push_ext(int np, int n, int expanding, double dtau, int step, double mass, const cplx *U,
                const double *Eo, const double *En, const double *phi, const double *pio,
                const double *pin, double *x, double *y, double *eta, double *px, double *py,
                double *peta, double *Q, const double *p0, double acc[4], int integrator, int substeps,
                int interp) {
    const double tau_n = step * dtau, h = dtau / substeps;
    double sx = 0, sy = 0, sz = 0;
#pragma omp parallel for reduction(+ : sx, sy, sz)
    for (int j = 0; j < np; j++) {
        double *q = Q + 8 * j;
        double xj = x[j], yj = y[j];
        double pk[3] = {px[j], py[j], peta[j]};
        for (int k = 0; k < substeps; k++) {
            const double tau_k = tau_n + k * h;
            const double te_h = expanding ? tau_k + 0.5 * h : 1.0;
            int cx = (int)floor(xj), cy = (int)floor(yj);
            double F[6][8];
            if (interp)
                o_gather_cic(n, tau_n, expanding, U, Eo, En, phi, pio, pin, cx, cy, xj - cx, yj - cy, F);
            else
                o_gather(n, tau_n, expanding, U, Eo, En, phi, pio, pin, cx, cy, F);
            double qE[3] = {dot8(q, F[0]), dot8(q, F[1]), dot8(q, F[2])};
            double qB[3] = {dot8(q, F[3]), dot8(q, F[4]), dot8(q, F[5])};
            kick(integrator, expanding, h, tau_k, mass, qE, qB, pk);
            double ptn = sqrt(mass * mass + pk[0] * pk[0] + pk[1] * pk[1] + pk[2] * pk[2]);
            double iptn = ptn > 0 ? 1.0 / ptn : 0.0;
            double xn = xj + h * pk[0] * iptn;
            double yn = yj + h * pk[1] * iptn;
            double deta = h * pk[2] * iptn / te_h;
            /* color: rotation along eta at the old cell */
            {
                double a[8];
                cplx W[9];
                for (int c = 0; c < 8; c++) a[c] = -phi[8 * site(n, cx, cy) + c] * deta;
                o_exp_i(a, W);
                double qn[8];
                o_conj_by(W, q, qn);
                memcpy(q, qn, sizeof(qn));
            }
            int nx = (int)floor(xn), ny = (int)floor(yn);
            double qn[8];
            if (nx == cx + 1) { o_transport(U + 18 * site(n, cx, cy) + 0, q, qn); memcpy(q, qn, sizeof(qn)); }
            else if (nx == cx - 1) { o_conj_by(U + 18 * site(n, cx - 1, cy) + 0, q, qn); memcpy(q, qn, sizeof(qn)); }
            if (ny == cy + 1) { o_transport(U + 18 * site(n, nx, cy) + 9, q, qn); memcpy(q, qn, sizeof(qn)); }
            else if (ny == cy - 1) { o_conj_by(U + 18 * site(n, nx, cy - 1) + 9, q, qn); memcpy(q, qn, sizeof(qn)); }
            /* periodic wrap, keeping x inside its cell */
            if (nx < 0) { xn += n; nx += n; } else if (nx >= n) { xn -= n; nx -= n; }
            if (ny < 0) { yn += n; ny += n; } else if (ny >= n) { yn -= n; ny -= n; }
            if (xn < nx) xn = nx;
            if (xn >= nx + 1) xn = nextafter((double)(nx + 1), 0.0);
            if (yn < ny) yn = ny;
            if (yn >= ny + 1) yn = nextafter((double)(ny + 1), 0.0);
            xj = xn; yj = yn;
            eta[j] += deta;
        }
        x[j] = xj; y[j] = yj;
        px[j] = pk[0]; py[j] = pk[1]; peta[j] = pk[2];
        double pz = expanding ? o_pz_lab(mass, pk[0], pk[1], pk[2], eta[j]) : pk[2];
        sx += pk[0] * pk[0] - p0[3 * j + 0] * p0[3 * j + 0];
        sy += pk[1] * pk[1] - p0[3 * j + 1] * p0[3 * j + 1];
        sz += pz * pz - p0[3 * j + 2] * p0[3 * j + 2];
    }
    acc[0] += sx;
    acc[1] += sy;
    acc[2] += sz;
    acc[3] += np;
}
