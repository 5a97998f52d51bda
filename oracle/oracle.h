/*
 * FP64 CPU oracle for the boost-invariant SU(3) Glasma + colored particle-in-cell
 * method of arXiv:2307.07999 (Avramescu et al., "Heavy quark kappa and jet qhat
 * transport coefficients in the Glasma early stage of heavy-ion collisions").
 *
 * THIS IS TEST INFRASTRUCTURE.  It is a plain, slow, obviously-correct restatement
 * of the method used only by the test-suite, by __graft_entry__.smoke() and by the
 * CPU-baseline leg of bench.py.  No product code path may call it.  It shares no
 * code, header, table or constant generator with the CUDA library in
 * paper_2307_07999_gb300/csrc; the two are compared element by element.
 *
 * Conventions (lattice units, a = 1, g absorbed into the fields):
 *   - N x N periodic transverse lattice, site index s = x + N*y.
 *   - t^a = lambda^a / 2 (Gell-Mann), Tr t^a t^b = delta^ab / 2.
 *   - Algebra elements X = X^a t^a are stored as 8 reals.
 *   - Complex 3x3 matrices are stored row-major as 9 complex = 18 doubles
 *     (re, im interleaved; C99 double complex layout).
 *   - U[s][d][9] (d = 0: x-link, d = 1: y-link), E[s][d][8], phi[s][8], pi[s][8].
 *   - Staggering: U, phi live at tau_n = n*dtau; E, pi live at tau_{n-1/2}.
 *
 * Parity status per function is given in the header comment of each .c file.
 */
#ifndef GLASMA_ORACLE_H
#define GLASMA_ORACLE_H
#include <stdint.h>
#include <complex.h>

typedef double complex cplx;

/* ---------------- su3.c : SU(3) algebra ---------------- */
void o_generator(int a, cplx T[9]);                     /* t^a, a = 0..7 */
void o_alg_to_mat(const double x[8], cplx X[9]);         /* X = x^a t^a */
void o_mat_to_alg(const cplx X[9], double x[8]);         /* x^a = 2 Re Tr(t^a X) */
void o_im_tl(const cplx P[9], double x[8]);              /* x^a = 2 Im Tr(t^a P) */
void o_mul(const cplx A[9], const cplx B[9], cplx C[9]); /* C = A B */
void o_dag(const cplx A[9], cplx B[9]);                  /* B = A^dagger */
void o_mul_dn(const cplx A[9], const cplx B[9], cplx C[9]); /* C = A B^dagger */
void o_mul_nd(const cplx A[9], const cplx B[9], cplx C[9]); /* C = A^dagger B */
void o_exp_i(const double x[8], cplx U[9]);              /* U = exp(i x^a t^a) */
void o_expm(const cplx A[9], cplx R[9]);                 /* R = exp(A), any 3x3 */
void o_transport(const cplx U[9], const double x[8], double y[8]); /* y = U^dag X U */
void o_conj_by(const cplx U[9], const double x[8], double y[8]);   /* y = U X U^dag */
void o_icomm(const double a[8], const double b[8], double c[8]);   /* c = i[A, B] */
void o_structure_constants(double f[512], double d[512]);
void o_haar(const double g[18], cplx U[9]);  /* U(3) Haar from 9 complex Gaussians */
void o_reunitarize(cplx U[9]);
double o_unitarity_dev(const cplx U[9]);    /* max |U U^dag - 1| and |det U - 1| */
cplx o_det(const cplx U[9]);

/* ---------------- philox.c : counter-based RNG (Salmon et al. SC'11) --- */
void o_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double o_u01(uint32_t r);                   /* (r + 0.5) * 2^-32, in (0,1) */
void o_box_muller(uint32_t r0, uint32_t r1, double *g0, double *g1);

/* ---------------- fft.c : mixed-radix complex FFT ---------------- */
int o_fft2(int n, cplx *a, int sign);       /* in-place n x n, unnormalised */

/* ---------------- ic.c : MV initial conditions ---------------- */
void o_mv_charges(int n, int n_sheets, double g2mua, uint64_t seed,
                  int nucleus, int sheet, double *rho);          /* rho[s][8] */
int o_poisson(int n, double m2, const double *rho, double *lam); /* lam[s][8] */
int o_wilson_line(int n, int n_sheets, double g2mua, double m_ir_a, uint64_t seed,
                  int nucleus, cplx *V);                          /* V[s][9] */
void o_pure_gauge_links(int n, const cplx *V, cplx *UA);         /* UA[s][2][9] */
void o_ic_residual(const cplx U1[9], const cplx U2[9], const cplx U[9], double r[8]);
void o_ic_jacobian(const cplx U1[9], const cplx U2[9], const cplx U[9], double J[64]);
int o_ic_solve_link(const cplx U1[9], const cplx U2[9], cplx U[9], double tol,
                    int max_iter, double *res_out);             /* returns iterations or -1 */
int o_ic_solve(int n, const cplx *U1, const cplx *U2, const cplx *U_start,
               double tol, int max_iter, cplx *U, int32_t *iters, double *res);
void o_pi0(int n, const cplx *U, const cplx *U1, const cplx *U2, double *pi);
int o_glasma_init(int n, int n_sheets, double g2mua, double m_ir_a, uint64_t seed,
                  double dtau, double tol, int max_iter,
                  cplx *U, double *E, double *phi, double *pi, int32_t *iters);

/* ---------------- field.c : boost-invariant leapfrog ---------------- */
double o_potential(int n, double tau, int expanding, const cplx *U, const double *phi);
void o_force(int n, double tau, int expanding, const cplx *U, const double *phi,
             double *fE, double *fpi);
void o_field_step(int n, int expanding, double dtau, int step,
                  const cplx *U, const double *E, const double *phi, const double *pi,
                  cplx *U2, double *E2, double *phi2, double *pi2);
void o_reunitarize_all(int n, cplx *U);
void o_gauss(int n, const cplx *U, const double *E, const double *phi, const double *pi,
             double *G);
double o_gauss_rel(int n, const cplx *U, const double *E, const double *phi,
                   const double *pi);
void o_energy(int n, double tau, int expanding, const cplx *U, const double *E,
              const double *phi, const double *pi, double out[4]);
double o_unitarity_all(int n, const cplx *U);

/* ---------------- particles.c : Wong equations via CPIC ---------------- */
void o_particles_init(int np, int n, double mass, int init_kind, double p_min,
                      double p_max, double q2, double q3, uint64_t seed,
                      double *x, double *y, double *eta, double *px, double *py,
                      double *peta, double *Q);
void o_q0_cartan(double q2, double q3, double Q0[8]);
void o_gather(int n, double tau, int expanding, const cplx *U, const double *Eo,
              const double *En, const double *phi, const double *pio,
              const double *pin, int cx, int cy, double F[6][8]);
void o_push(int np, int n, int expanding, double dtau, int step, double mass,
            const cplx *U, const double *Eo, const double *En, const double *phi,
            const double *pio, const double *pin,
            double *x, double *y, double *eta, double *px, double *py, double *peta,
            double *Q, const double *p0, double acc[4]);
/* o_push with the integrator of the momentum kick: 0 explicit, 1 Boris */
void o_push_int(int np, int n, int expanding, double dtau, int step, double mass,
                const cplx *U, const double *Eo, const double *En, const double *phi,
                const double *pio, const double *pin,
                double *x, double *y, double *eta, double *px, double *py, double *peta,
                double *Q, const double *p0, double acc[4], int integrator);
/* cloud-in-cell gather: site-centred fields of c, c+x, c+y, c+x+y transported to c, bilinear weights */
void o_gather_cic(int n, double tau, int expanding, const cplx *U, const double *Eo, const double *En,
                  const double *phi, const double *pio, const double *pin, int cx, int cy, double ox,
                  double oy, double F[6][8]);
/* o_push_sub with interp: 0 nearest grid point, 1 cloud in cell */
void o_push_ext(int np, int n, int expanding, double dtau, int step, double mass,
                const cplx *U, const double *Eo, const double *En, const double *phi,
                const double *pio, const double *pin,
                double *x, double *y, double *eta, double *px, double *py, double *peta,
                double *Q, const double *p0, double acc[4], int integrator, int substeps, int interp);
/* o_push_int taken as `substeps` particle steps of dtau / substeps with the fields of the step */
void o_push_sub(int np, int n, int expanding, double dtau, int step, double mass,
                const cplx *U, const double *Eo, const double *En, const double *phi,
                const double *pio, const double *pin,
                double *x, double *y, double *eta, double *px, double *py, double *peta,
                double *Q, const double *p0, double acc[4], int integrator, int substeps);
void o_casimirs(const double Q[8], double *q2, double *q3);
/* OpenMP threads of the oracle's loops (timing only); returns the count in effect */
int o_set_threads(int n);
double o_pz_lab(double mass, double px, double py, double peta, double eta);

/* ---------------- correlators.c : Eqs. 4 and 5 ---------------- */
/* one step of the static (Istat[s][3][8]) and lightlike (W[s][9], J[s][3][8])
 * estimators; out = {<dp_x^2>, <dp_y^2>, <dp_z^2>} static, then lightlike */
void o_corr_step(int n, int expanding, double dtau, int step, const cplx *U, const double *Eo,
                 const double *En, const double *phi, const double *pio, const double *pin,
                 double *Istat, cplx *W, double *J, int k_now, int k_next, double out[6]);

/* ---------------- estimators.c : Eq. 3 transport coefficients ---------------- */
/* d f / d tau on the table's tau grid: central inside, one-sided at the ends */
void o_derivative(int rows, const double *tau, int tstride, const double *f, int fstride, double *df,
                  int dstride);
/* tab rows {tau, <dpx^2>, <dpy^2>, <dpz^2>, ...} (stride doubles); kind 0 heavy quarks,
 * 1 jets along x; out rows {tau, d/dtau of the three, transverse, longitudinal, total,
 * anisotropy} (8 doubles) */
void o_transport_coefficients(int rows, const double *tab, int stride, int kind, double *out);

/* ---------------- mlp.c : learned warm-start network ---------------- */
void o_mlp_forward(int batch, const double *x, const double *W1, const double *b1,
                   const double *W2, const double *b2, const double *W3,
                   const double *b3, double *h1, double *h2, double *y);
double o_mlp_loss_backward(int batch, const double *x, const double *target,
                           const double *W1, const double *b1, const double *W2,
                           const double *b2, const double *W3, const double *b3,
                           double *gW1, double *gb1, double *gW2, double *gb2,
                           double *gW3, double *gb3);
void o_ic_features(const cplx U1[9], const cplx U2[9], double feat[36]);
void o_ic_series(const cplx U1[9], const cplx U2[9], double ds[8]);
void o_ic_delta(const cplx U1[9], const cplx U2[9], const cplx U[9], double delta[8]);
void o_ic_target(const cplx U1[9], const cplx U2[9], const cplx U[9], double target[8]);

#endif
