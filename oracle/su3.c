/*
 * SU(3) algebra for the FP64 oracle (test infrastructure; see oracle.h).
 *
 * Everything here is the textbook definition written out with explicit
 * Gell-Mann matrices and traces.  The color charge Q = Q^a T^a and the
 * Casimirs q2 = Q^a Q^a, q3 = d_abc Q^a Q^b Q^c follow Sec. 1 ("Probes in
 * Glasma") of the paper; the group elements are the lattice gauge links of
 * Sec. 1 ("Glasma").  The matrix exponential is the scaling-and-squaring
 * Taylor method (Moler & Van Loan, "Nineteen dubious ways to compute the
 * exponential of a matrix", SIAM Review 2003, method 3 + squaring).
 * Haar-random U(3) elements follow Mezzadri, "How to generate random matrices
 * from the classical compact groups", Notices AMS 54 (2007): Gram-Schmidt of a
 * complex Ginibre matrix (R has positive diagonal, so no phase fix is needed).
 *
 * Pins (tests/test_oracle_su3.py): generator orthonormality and commutators,
 * f/d tables against the closed-form values (f123 = 1, d118 = 1/sqrt3, ...),
 * exp against scipy.linalg.expm and the abelian closed form, Haar moments,
 * reunitarisation of a perturbed matrix.
 */
#include <math.h>
#include <string.h>
#include "oracle.h"

static int gen_ready = 0;
static cplx T[8][9];

static void init_generators(void) {
    if (gen_ready) return;
    memset(T, 0, sizeof(T));
    const double h = 0.5;
    /* lambda_1 .. lambda_8, divided by 2 */
    T[0][1] = h;        T[0][3] = h;
    T[1][1] = -I * h;   T[1][3] = I * h;
    T[2][0] = h;        T[2][4] = -h;
    T[3][2] = h;        T[3][6] = h;
    T[4][2] = -I * h;   T[4][6] = I * h;
    T[5][5] = h;        T[5][7] = h;
    T[6][5] = -I * h;   T[6][7] = I * h;
    T[7][0] = h / sqrt(3.0); T[7][4] = h / sqrt(3.0); T[7][8] = -2.0 * h / sqrt(3.0);
    gen_ready = 1;
}

__attribute__((constructor)) static void su3_load_init(void) { init_generators(); }

void o_generator(int a, cplx out[9]) {
    init_generators();
    memcpy(out, T[a], sizeof(cplx) * 9);
}

static cplx trace_prod(const cplx A[9], const cplx B[9]) {
    cplx t = 0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) t += A[3 * i + j] * B[3 * j + i];
    return t;
}

void o_alg_to_mat(const double x[8], cplx X[9]) {
    init_generators();
    for (int k = 0; k < 9; k++) X[k] = 0;
    for (int a = 0; a < 8; a++)
        for (int k = 0; k < 9; k++) X[k] += x[a] * T[a][k];
}

void o_mat_to_alg(const cplx X[9], double x[8]) {
    init_generators();
    for (int a = 0; a < 8; a++) x[a] = 2.0 * creal(trace_prod(T[a], X));
}

void o_im_tl(const cplx P[9], double x[8]) {
    init_generators();
    for (int a = 0; a < 8; a++) x[a] = 2.0 * cimag(trace_prod(T[a], P));
}

void o_mul(const cplx A[9], const cplx B[9], cplx C[9]) {
    cplx R[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            cplx s = 0;
            for (int k = 0; k < 3; k++) s += A[3 * i + k] * B[3 * k + j];
            R[3 * i + j] = s;
        }
    memcpy(C, R, sizeof(R));
}

void o_dag(const cplx A[9], cplx B[9]) {
    cplx R[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) R[3 * i + j] = conj(A[3 * j + i]);
    memcpy(B, R, sizeof(R));
}

void o_mul_dn(const cplx A[9], const cplx B[9], cplx C[9]) {
    cplx Bd[9];
    o_dag(B, Bd);
    o_mul(A, Bd, C);
}

void o_mul_nd(const cplx A[9], const cplx B[9], cplx C[9]) {
    cplx Ad[9];
    o_dag(A, Ad);
    o_mul(Ad, B, C);
}

static double fro(const cplx A[9]) {
    double s = 0;
    for (int k = 0; k < 9; k++) s += creal(A[k] * conj(A[k]));
    return sqrt(s);
}

void o_expm(const cplx A[9], cplx R[9]) {
    /* scaling: ||A / 2^s||_F <= 1/4 */
    double nrm = fro(A);
    int s = 0;
    while (nrm > 0.25) { nrm *= 0.5; s++; }
    double scale = ldexp(1.0, -s);
    cplx B[9], term[9], sum[9];
    for (int k = 0; k < 9; k++) B[k] = A[k] * scale;
    for (int k = 0; k < 9; k++) { term[k] = (k % 4 == 0) ? 1.0 : 0.0; sum[k] = term[k]; }
    for (int n = 1; n <= 40; n++) {
        o_mul(term, B, term);
        for (int k = 0; k < 9; k++) term[k] /= (double)n;
        for (int k = 0; k < 9; k++) sum[k] += term[k];
        if (fro(term) < 1e-22) break;
    }
    for (int i = 0; i < s; i++) o_mul(sum, sum, sum);
    memcpy(R, sum, sizeof(sum));
}

void o_exp_i(const double x[8], cplx U[9]) {
    cplx X[9];
    o_alg_to_mat(x, X);
    for (int k = 0; k < 9; k++) X[k] *= I;
    o_expm(X, U);
}

void o_transport(const cplx U[9], const double x[8], double y[8]) {
    cplx X[9], t[9];
    o_alg_to_mat(x, X);
    o_mul_nd(U, X, t);   /* U^dag X */
    o_mul(t, U, t);      /* U^dag X U */
    o_mat_to_alg(t, y);
}

void o_conj_by(const cplx U[9], const double x[8], double y[8]) {
    cplx X[9], t[9];
    o_alg_to_mat(x, X);
    o_mul(U, X, t);      /* U X */
    o_mul_dn(t, U, t);   /* U X U^dag */
    o_mat_to_alg(t, y);
}

void o_structure_constants(double f[512], double d[512]) {
    init_generators();
    cplx ab[9], ba[9], c1[9], c2[9];
    for (int a = 0; a < 8; a++)
        for (int b = 0; b < 8; b++) {
            o_mul(T[a], T[b], ab);
            o_mul(T[b], T[a], ba);
            for (int k = 0; k < 9; k++) { c1[k] = ab[k] - ba[k]; c2[k] = ab[k] + ba[k]; }
            for (int c = 0; c < 8; c++) {
                /* [t^a, t^b] = i f^abc t^c ; {t^a, t^b} = delta/3 + d^abc t^c */
                f[64 * a + 8 * b + c] = creal(-2.0 * I * trace_prod(c1, T[c]));
                d[64 * a + 8 * b + c] = creal(2.0 * trace_prod(c2, T[c]));
            }
        }
}

void o_haar(const double g[18], cplx U[9]) {
    cplx Z[9];
    for (int k = 0; k < 9; k++) Z[k] = (g[2 * k] + I * g[2 * k + 1]) / sqrt(2.0);
    /* modified Gram-Schmidt on the columns */
    for (int j = 0; j < 3; j++) {
        cplx v[3] = {Z[j], Z[3 + j], Z[6 + j]};
        for (int k = 0; k < j; k++) {
            cplx ip = 0;
            for (int i = 0; i < 3; i++) ip += conj(U[3 * i + k]) * v[i];
            for (int i = 0; i < 3; i++) v[i] -= ip * U[3 * i + k];
        }
        double nv = 0;
        for (int i = 0; i < 3; i++) nv += creal(v[i] * conj(v[i]));
        nv = sqrt(nv);
        for (int i = 0; i < 3; i++) U[3 * i + j] = v[i] / nv;
    }
}

void o_reunitarize(cplx U[9]) {
    cplx *r1 = U, *r2 = U + 3, *r3 = U + 6;
    double n1 = 0;
    for (int k = 0; k < 3; k++) n1 += creal(r1[k] * conj(r1[k]));
    n1 = sqrt(n1);
    for (int k = 0; k < 3; k++) r1[k] /= n1;
    cplx ip = 0;
    for (int k = 0; k < 3; k++) ip += conj(r1[k]) * r2[k];
    for (int k = 0; k < 3; k++) r2[k] -= ip * r1[k];
    double n2 = 0;
    for (int k = 0; k < 3; k++) n2 += creal(r2[k] * conj(r2[k]));
    n2 = sqrt(n2);
    for (int k = 0; k < 3; k++) r2[k] /= n2;
    /* third row = complex conjugate of the cross product r1 x r2 (det = 1) */
    r3[0] = conj(r1[1] * r2[2] - r1[2] * r2[1]);
    r3[1] = conj(r1[2] * r2[0] - r1[0] * r2[2]);
    r3[2] = conj(r1[0] * r2[1] - r1[1] * r2[0]);
}

cplx o_det(const cplx U[9]) {
    return U[0] * (U[4] * U[8] - U[5] * U[7]) - U[1] * (U[3] * U[8] - U[5] * U[6]) +
           U[2] * (U[3] * U[7] - U[4] * U[6]);
}

double o_unitarity_dev(const cplx U[9]) {
    cplx P[9];
    o_mul_dn(U, U, P);
    double m = 0;
    for (int k = 0; k < 9; k++) {
        double v = cabs(P[k] - ((k % 4 == 0) ? 1.0 : 0.0));
        if (v > m) m = v;
    }
    double dd = cabs(o_det(U) - 1.0);
    return dd > m ? dd : m;
}

/* components of i[A, B] for Hermitian A = a^a t^a, B = b^a t^a */
void o_icomm(const double a[8], const double b[8], double out[8]) {
    cplx A[9], B[9], AB[9], BA[9], C[9];
    o_alg_to_mat(a, A);
    o_alg_to_mat(b, B);
    o_mul(A, B, AB);
    o_mul(B, A, BA);
    for (int k = 0; k < 9; k++) C[k] = I * (AB[k] - BA[k]);
    o_mat_to_alg(C, out);
}

/* Threads of the OpenMP loops (timing the oracle on one core or all cores; no effect
 * without OpenMP).  Returns the count in effect. */
#ifdef _OPENMP
#include <omp.h>
#endif
int o_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
