// SU(3) / su(3) device arithmetic for the GB300 Glasma + CPIC library.
//
// Conventions (Sec. 1 of arXiv:2307.07999, lattice units, g absorbed):
//   t^a = lambda^a / 2, algebra elements X = X^a t^a stored as 8 reals,
//   links U in SU(3); only rows 0 and 1 are stored, row 2 = conj(r0 x r1).
// Everything here is written for register-resident 3x3 blocks: Hermitian
// matrices keep their 3 real diagonal and 3 complex upper entries, the
// exponential uses the Cayley-Hamilton reduction X^3 = c1 X + c0 1 of a
// traceless 3x3 matrix (c1 = Tr X^2 / 2, c0 = det X) so the Taylor series runs
// on three complex scalars, and commutators use the SU(3) structure constants
// f^abc (standard Gell-Mann table).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define DEV __device__ __forceinline__

namespace glasma {

template <class T> struct cx { T r, i; };
template <class T> DEV cx<T> mk(T r, T i) { cx<T> z; z.r = r; z.i = i; return z; }
template <class T> DEV cx<T> operator+(cx<T> a, cx<T> b) { return mk(a.r + b.r, a.i + b.i); }
template <class T> DEV cx<T> operator-(cx<T> a, cx<T> b) { return mk(a.r - b.r, a.i - b.i); }
template <class T> DEV cx<T> operator*(cx<T> a, cx<T> b) {
    return mk(a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r);
}
template <class T> DEV cx<T> operator*(T s, cx<T> a) { return mk(s * a.r, s * a.i); }
template <class T> DEV cx<T> cj(cx<T> a) { return mk(a.r, -a.i); }
// a * conj(b)
template <class T> DEV cx<T> mulc(cx<T> a, cx<T> b) {
    return mk(a.r * b.r + a.i * b.i, a.i * b.r - a.r * b.i);
}
// acc += a * b
template <class T> DEV void fma_(cx<T>& acc, cx<T> a, cx<T> b) {
    acc.r = fma(a.r, b.r, fma(-a.i, b.i, acc.r));
    acc.i = fma(a.r, b.i, fma(a.i, b.r, acc.i));
}
// acc += a * conj(b)
template <class T> DEV void fmac_(cx<T>& acc, cx<T> a, cx<T> b) {
    acc.r = fma(a.r, b.r, fma(a.i, b.i, acc.r));
    acc.i = fma(a.i, b.r, fma(-a.r, b.i, acc.i));
}
// acc += conj(a) * b
template <class T> DEV void fmca_(cx<T>& acc, cx<T> a, cx<T> b) {
    acc.r = fma(a.r, b.r, fma(a.i, b.i, acc.r));
    acc.i = fma(a.r, b.i, fma(-a.i, b.r, acc.i));
}

// ---------------------------------------------------------------- complex products
// Accumulated complex products.  In FP32 they run on the sm_100-family paired FMA
// (fma.rn.f32x2) with the complex number as the register pair (re, im):
//   a b       = a.r (b.r, b.i) + a.i (-b.i, b.r)
//   a conj(b) = a.r (b.r, -b.i) + a.i (b.i, b.r)
//   conj(a) b = a.r (b.r, b.i) + a.i (b.i, -b.r)
// two paired FMAs where the scalar form takes four (the broadcast pairs (a.r, a.r)
// cost nothing; a negated lane costs one instruction, shared by every product that
// reuses b).  FP64 keeps scalar FMAs.
template <class T> struct CA;
template <> struct CA<double> { cx<double> z; };
template <> struct CA<float> { unsigned long long v; };

DEV unsigned long long pk2(float a, float b) {
    unsigned long long d;
    asm("mov.b64 %0, {%1,%2};" : "=l"(d) : "f"(a), "f"(b));
    return d;
}
DEV cx<float> upk2(unsigned long long d) {
    cx<float> z;
    asm("mov.b64 {%0,%1}, %2;" : "=f"(z.r), "=f"(z.i) : "l"(d));
    return z;
}
DEV unsigned long long ffma2(unsigned long long a, unsigned long long b, unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
DEV unsigned long long fmul2(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
DEV unsigned long long fadd2(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
DEV unsigned long long fsub2(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

DEV cx<float> val(CA<float> a) { return upk2(a.v); }
DEV cx<double> val(CA<double> a) { return a.z; }
// a b
DEV CA<float> cmul(cx<float> a, cx<float> b) {
    return {ffma2(pk2(a.i, a.i), pk2(-b.i, b.r), fmul2(pk2(a.r, a.r), pk2(b.r, b.i)))};
}
DEV CA<double> cmul(cx<double> a, cx<double> b) { return {a * b}; }
// acc + a b
DEV CA<float> cmac(CA<float> c, cx<float> a, cx<float> b) {
    return {ffma2(pk2(a.i, a.i), pk2(-b.i, b.r), ffma2(pk2(a.r, a.r), pk2(b.r, b.i), c.v))};
}
DEV CA<double> cmac(CA<double> c, cx<double> a, cx<double> b) { fma_(c.z, a, b); return c; }
// a conj(b)
DEV CA<float> cmulc(cx<float> a, cx<float> b) {
    return {ffma2(pk2(a.i, a.i), pk2(b.i, b.r), fmul2(pk2(a.r, a.r), pk2(b.r, -b.i)))};
}
DEV CA<double> cmulc(cx<double> a, cx<double> b) { return {mulc(a, b)}; }
// acc + a conj(b)
DEV CA<float> cmacc(CA<float> c, cx<float> a, cx<float> b) {
    return {ffma2(pk2(a.i, a.i), pk2(b.i, b.r), ffma2(pk2(a.r, a.r), pk2(b.r, -b.i), c.v))};
}
DEV CA<double> cmacc(CA<double> c, cx<double> a, cx<double> b) { fmac_(c.z, a, b); return c; }
// conj(a) b
DEV CA<float> ccmul(cx<float> a, cx<float> b) {
    return {ffma2(pk2(a.i, a.i), pk2(b.i, -b.r), fmul2(pk2(a.r, a.r), pk2(b.r, b.i)))};
}
DEV CA<double> ccmul(cx<double> a, cx<double> b) { return {mk(a.r * b.r + a.i * b.i, a.r * b.i - a.i * b.r)}; }
// acc + conj(a) b
DEV CA<float> ccmac(CA<float> c, cx<float> a, cx<float> b) {
    return {ffma2(pk2(a.i, a.i), pk2(b.i, -b.r), ffma2(pk2(a.r, a.r), pk2(b.r, b.i), c.v))};
}
DEV CA<double> ccmac(CA<double> c, cx<double> a, cx<double> b) { fmca_(c.z, a, b); return c; }
// s b and acc + s b for real s
DEV CA<float> rmul(float s, cx<float> b) { return {fmul2(pk2(s, s), pk2(b.r, b.i))}; }
DEV CA<double> rmul(double s, cx<double> b) { return {s * b}; }
DEV CA<float> rmac(CA<float> c, float s, cx<float> b) { return {ffma2(pk2(s, s), pk2(b.r, b.i), c.v)}; }
DEV CA<double> rmac(CA<double> c, double s, cx<double> b) {
    c.z.r = fma(s, b.r, c.z.r);
    c.z.i = fma(s, b.i, c.z.i);
    return c;
}
// Re(conj(a) b) summed over three pairs: the real part of a Hermitian product's diagonal
DEV float redot3(cx<float> a0, cx<float> b0, cx<float> a1, cx<float> b1, cx<float> a2, cx<float> b2) {
    const cx<float> p = upk2(ffma2(pk2(a2.r, a2.i), pk2(b2.r, b2.i),
                                   ffma2(pk2(a1.r, a1.i), pk2(b1.r, b1.i), fmul2(pk2(a0.r, a0.i), pk2(b0.r, b0.i)))));
    return p.r + p.i;
}
DEV double redot3(cx<double> a0, cx<double> b0, cx<double> a1, cx<double> b1, cx<double> a2, cx<double> b2) {
    return fma(a2.r, b2.r, fma(a2.i, b2.i, fma(a1.r, b1.r, fma(a1.i, b1.i, fma(a0.r, b0.r, a0.i * b0.i)))));
}

template <class T> struct M3 { cx<T> m[3][3]; };   // general 3x3 complex
template <class T> struct Al { T a[8]; };          // su(3) components
// Hermitian 3x3: real diagonal d0,d1,d2 and upper entries u01,u02,u12
template <class T> struct H3 { T d0, d1, d2; cx<T> u01, u02, u12; };

template <class T> DEV T inv_sqrt3() { return T(0.57735026918962576451); }

// ---------------------------------------------------------------- conversions
template <class T> DEV H3<T> herm(const Al<T>& x) {
    const T h = T(0.5), s = h * inv_sqrt3<T>();
    H3<T> X;
    X.d0 = h * x.a[2] + s * x.a[7];
    X.d1 = -h * x.a[2] + s * x.a[7];
    X.d2 = T(-2) * s * x.a[7];
    X.u01 = mk(h * x.a[0], -h * x.a[1]);
    X.u02 = mk(h * x.a[3], -h * x.a[4]);
    X.u12 = mk(h * x.a[5], -h * x.a[6]);
    return X;
}
template <class T> DEV Al<T> alg(const H3<T>& X) {
    Al<T> x;
    x.a[0] = T(2) * X.u01.r;  x.a[1] = T(-2) * X.u01.i;
    x.a[2] = X.d0 - X.d1;
    x.a[3] = T(2) * X.u02.r;  x.a[4] = T(-2) * X.u02.i;
    x.a[5] = T(2) * X.u12.r;  x.a[6] = T(-2) * X.u12.i;
    x.a[7] = (X.d0 + X.d1 - T(2) * X.d2) * inv_sqrt3<T>();
    return x;
}
template <class T> DEV cx<T> hget(const H3<T>& X, int i, int j) {
    if (i == j) return mk(i == 0 ? X.d0 : (i == 1 ? X.d1 : X.d2), T(0));
    if (i == 0 && j == 1) return X.u01;
    if (i == 0 && j == 2) return X.u02;
    if (i == 1 && j == 2) return X.u12;
    if (i == 1 && j == 0) return cj(X.u01);
    if (i == 2 && j == 0) return cj(X.u02);
    return cj(X.u12);
}
// components of ImTL(P) = [(P - P^dag)/(2i)]_traceless : x^a = 2 Im Tr(t^a P)
template <class T> DEV Al<T> im_tl(const M3<T>& P) {
    Al<T> x;
    x.a[0] = P.m[0][1].i + P.m[1][0].i;
    x.a[1] = P.m[0][1].r - P.m[1][0].r;
    x.a[2] = P.m[0][0].i - P.m[1][1].i;
    x.a[3] = P.m[0][2].i + P.m[2][0].i;
    x.a[4] = P.m[0][2].r - P.m[2][0].r;
    x.a[5] = P.m[1][2].i + P.m[2][1].i;
    x.a[6] = P.m[1][2].r - P.m[2][1].r;
    x.a[7] = (P.m[0][0].i + P.m[1][1].i - T(2) * P.m[2][2].i) * inv_sqrt3<T>();
    return x;
}

// ---------------------------------------------------------------- links
// row 2 of an SU(3) matrix from rows 0 and 1
template <class T> DEV void complete_row2(M3<T>& U) {
    const cx<T>* a = U.m[0];
    const cx<T>* b = U.m[1];
    U.m[2][0] = cj(val(cmul(a[1], b[2])) - val(cmul(a[2], b[1])));
    U.m[2][1] = cj(val(cmul(a[2], b[0])) - val(cmul(a[0], b[2])));
    U.m[2][2] = cj(val(cmul(a[0], b[1])) - val(cmul(a[1], b[0])));
}
// C = A B
template <class T> DEV M3<T> mul(const M3<T>& A, const M3<T>& B) {
    M3<T> C;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++)
            C.m[i][j] = val(cmac(cmac(cmul(A.m[i][0], B.m[0][j]), A.m[i][1], B.m[1][j]), A.m[i][2], B.m[2][j]));
    return C;
}
// C = A B^dag
template <class T> DEV M3<T> mul_nd(const M3<T>& A, const M3<T>& B) {
    M3<T> C;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++)
            C.m[i][j] = val(cmacc(cmacc(cmulc(A.m[i][0], B.m[j][0]), A.m[i][1], B.m[j][1]), A.m[i][2], B.m[j][2]));
    return C;
}
// ImTL(A B^dag) without forming the real parts of the diagonal
template <class T> DEV Al<T> im_tl_nd(const M3<T>& A, const M3<T>& B) {
    return im_tl(mul_nd(A, B));
}

// (X B)_ij for Hermitian X: sum_k X_ik B_kj with X_ik real on the diagonal, the
// stored upper entry above it and its conjugate below
template <class T> DEV cx<T> hmul_entry(const H3<T>& X, const M3<T>& B, int i, int j) {
    if (i == 0) return val(cmac(cmac(rmul(X.d0, B.m[0][j]), X.u01, B.m[1][j]), X.u02, B.m[2][j]));
    if (i == 1) return val(cmac(rmac(ccmul(X.u01, B.m[0][j]), X.d1, B.m[1][j]), X.u12, B.m[2][j]));
    return val(rmac(ccmac(ccmul(X.u02, B.m[0][j]), X.u12, B.m[1][j]), X.d2, B.m[2][j]));
}
// (A X)_ij for Hermitian X
template <class T> DEV cx<T> mulh_entry(const M3<T>& A, const H3<T>& X, int i, int j) {
    if (j == 0) return val(cmacc(cmacc(rmul(X.d0, A.m[i][0]), A.m[i][1], X.u01), A.m[i][2], X.u02));
    if (j == 1) return val(cmacc(rmac(cmul(A.m[i][0], X.u01), X.d1, A.m[i][1]), A.m[i][2], X.u12));
    return val(rmac(cmac(cmul(A.m[i][0], X.u02), A.m[i][1], X.u12), X.d2, A.m[i][2]));
}
// U^dag X U for Hermitian X (result Hermitian; only diagonal + upper computed)
template <class T> DEV H3<T> transport(const M3<T>& U, const H3<T>& X) {
    M3<T> W;  // X U
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) W.m[i][j] = hmul_entry(X, U, i, j);
    // R_ij = sum_k conj(U_ki) W_kj
    H3<T> R;
    R.d0 = redot3(U.m[0][0], W.m[0][0], U.m[1][0], W.m[1][0], U.m[2][0], W.m[2][0]);
    R.d1 = redot3(U.m[0][1], W.m[0][1], U.m[1][1], W.m[1][1], U.m[2][1], W.m[2][1]);
    R.d2 = redot3(U.m[0][2], W.m[0][2], U.m[1][2], W.m[1][2], U.m[2][2], W.m[2][2]);
    R.u01 = val(ccmac(ccmac(ccmul(U.m[0][0], W.m[0][1]), U.m[1][0], W.m[1][1]), U.m[2][0], W.m[2][1]));
    R.u02 = val(ccmac(ccmac(ccmul(U.m[0][0], W.m[0][2]), U.m[1][0], W.m[1][2]), U.m[2][0], W.m[2][2]));
    R.u12 = val(ccmac(ccmac(ccmul(U.m[0][1], W.m[0][2]), U.m[1][1], W.m[1][2]), U.m[2][1], W.m[2][2]));
    return R;
}
// U X U^dag for Hermitian X
template <class T> DEV H3<T> conj_by(const M3<T>& U, const H3<T>& X) {
    M3<T> W;  // U X
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) W.m[i][j] = mulh_entry(U, X, i, j);
    // R_ij = sum_k W_ik conj(U_jk)
    H3<T> R;
    R.d0 = redot3(U.m[0][0], W.m[0][0], U.m[0][1], W.m[0][1], U.m[0][2], W.m[0][2]);
    R.d1 = redot3(U.m[1][0], W.m[1][0], U.m[1][1], W.m[1][1], U.m[1][2], W.m[1][2]);
    R.d2 = redot3(U.m[2][0], W.m[2][0], U.m[2][1], W.m[2][1], U.m[2][2], W.m[2][2]);
    R.u01 = val(cmacc(cmacc(cmulc(W.m[0][0], U.m[1][0]), W.m[0][1], U.m[1][1]), W.m[0][2], U.m[1][2]));
    R.u02 = val(cmacc(cmacc(cmulc(W.m[0][0], U.m[2][0]), W.m[0][1], U.m[2][1]), W.m[0][2], U.m[2][2]));
    R.u12 = val(cmacc(cmacc(cmulc(W.m[1][0], U.m[2][0]), W.m[1][1], U.m[2][1]), W.m[1][2], U.m[2][2]));
    return R;
}
template <class T> DEV Al<T> transport_alg(const M3<T>& U, const Al<T>& x) {
    return alg(transport(U, herm(x)));
}
template <class T> DEV Al<T> conj_alg(const M3<T>& U, const Al<T>& x) {
    return alg(conj_by(U, herm(x)));
}

// i[A, B] in components: (i[A,B])^c = -f^abc A^a B^b.  Independent nonzero f
// (1-based): f123 = 1, f147 = f246 = f257 = f345 = 1/2, f156 = f367 = -1/2,
// f458 = f678 = sqrt(3)/2.
template <class T> DEV Al<T> icomm(const Al<T>& A, const Al<T>& B) {
    Al<T> c;
#pragma unroll
    for (int k = 0; k < 8; k++) c.a[k] = T(0);
    const T h = T(0.5), r = T(0.86602540378443864676);
#define GL_F(p, q, s, v)                                             \
    c.a[s] -= (v) * (A.a[p] * B.a[q] - A.a[q] * B.a[p]);             \
    c.a[p] -= (v) * (A.a[q] * B.a[s] - A.a[s] * B.a[q]);             \
    c.a[q] -= (v) * (A.a[s] * B.a[p] - A.a[p] * B.a[s]);
    GL_F(0, 1, 2, T(1))
    GL_F(0, 3, 6, h)
    GL_F(0, 4, 5, -h)
    GL_F(1, 3, 5, h)
    GL_F(1, 4, 6, h)
    GL_F(2, 3, 4, h)
    GL_F(2, 5, 6, -h)
    GL_F(3, 4, 7, r)
    GL_F(5, 6, 7, r)
#undef GL_F
    return c;
}

// ---------------------------------------------------------------- exponential
// Hermitian square
template <class T> DEV H3<T> hsq(const H3<T>& X) {
    H3<T> Y;
    const cx<T> a = X.u01, b = X.u02, c = X.u12;
    const T na = a.r * a.r + a.i * a.i, nb = b.r * b.r + b.i * b.i, nc = c.r * c.r + c.i * c.i;
    Y.d0 = X.d0 * X.d0 + na + nb;
    Y.d1 = X.d1 * X.d1 + na + nc;
    Y.d2 = X.d2 * X.d2 + nb + nc;
    // (X^2)_01 = d0 a + a d1 + b conj(c)
    Y.u01 = (X.d0 + X.d1) * a + mulc(b, c);
    // (X^2)_02 = d0 b + a c + b d2
    Y.u02 = (X.d0 + X.d2) * b + a * c;
    // (X^2)_12 = conj(a) b + d1 c + c d2
    Y.u12 = (X.d1 + X.d2) * c + cj(a) * b;
    return Y;
}
template <class T> DEV T hdet(const H3<T>& X) {
    const cx<T> a = X.u01, b = X.u02, c = X.u12;
    const T na = a.r * a.r + a.i * a.i, nb = b.r * b.r + b.i * b.i, nc = c.r * c.r + c.i * c.i;
    const cx<T> acb = mulc(a * c, b);  // a c conj(b)
    return X.d0 * X.d1 * X.d2 - X.d0 * nc - X.d1 * nb - X.d2 * na + T(2) * acb.r;
}

// Taylor terms after scaling to ||X||_F <= 1/2 (eigenvalues <= 0.41): the remainder
// 0.41^(K+1)/(K+1)! is 2e-8 for K = 7 (below FP32 rounding) and 1e-19 for K = 16.
template <class T> struct ExpTerms { static constexpr int K = 16; };
template <> struct ExpTerms<float> { static constexpr int K = 7; };

// exp(i X) for Hermitian traceless X, returned as W = f0 1 + f1 X + f2 X^2
template <class T> DEV M3<T> expi(const H3<T>& X) {
    const H3<T> X2 = hsq(X);
    const T c1 = T(0.5) * (X2.d0 + X2.d1 + X2.d2);
    const T c0 = hdet(X);
    // scale so that ||X / 2^s||_F^2 = 2 c1 / 4^s <= 1/4
    int s = 0;
    T n2 = T(2) * c1;
    while (n2 > T(0.25) && s < 40) { n2 *= T(0.25); s++; }
    const T sc = ldexp(T(1), -s);
    const T c1s = c1 * sc * sc, c0s = c0 * sc * sc * sc;
    // Y^k = a I + b Y + d Y^2 ;  exp(iY) = sum_k i^k/k! Y^k
    T a = T(0), b = T(0), d = T(1);  // Y^2
    cx<T> f0 = mk(T(1), T(0)), f1 = mk(T(0), T(1)), f2 = mk(T(-0.5), T(0));
    T coef = T(0.5);  // 1/k!
#pragma unroll
    for (int k = 3; k <= ExpTerms<T>::K; k++) {
        const T na = c0s * d, nb = a + c1s * d, nd = b;
        a = na; b = nb; d = nd;
        coef /= T(k);
        // i^k: k mod 4 = 0: 1, 1: i, 2: -1, 3: -i
        const int m = k & 3;
        const T sr = (m == 0) ? coef : ((m == 2) ? -coef : T(0));
        const T si = (m == 1) ? coef : ((m == 3) ? -coef : T(0));
        f0.r += sr * a; f0.i += si * a;
        f1.r += sr * b; f1.i += si * b;
        f2.r += sr * d; f2.i += si * d;
    }
    for (int q = 0; q < s; q++) {
        const cx<T> f12 = f1 * f2, f22 = f2 * f2;
        const cx<T> g0 = f0 * f0 + (T(2) * c0s) * f12;
        const cx<T> g1 = T(2) * (f0 * f1) + (T(2) * c1s) * f12 + c0s * f22;
        const cx<T> g2 = T(2) * (f0 * f2) + f1 * f1 + c1s * f22;
        f0 = g0; f1 = g1; f2 = g2;
    }
    // back to the basis {1, X, X^2}
    f1 = sc * f1;
    f2 = (sc * sc) * f2;
    M3<T> W;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            cx<T> w;
            if (i == j) w = val(rmac(rmul(hget(X, i, i).r, f1), hget(X2, i, i).r, f2)) + f0;
            else if (i < j) w = val(cmac(cmul(f1, hget(X, i, j)), f2, hget(X2, i, j)));
            else w = val(cmacc(cmulc(f1, hget(X, j, i)), f2, hget(X2, j, i)));
            W.m[i][j] = w;
        }
    return W;
}

// Renormalisation of rows 0, 1 in the working precision, for links within rounding of
// SU(3): with |r|^2 = 1 + d, the Newton step r <- r - (d / 2) r leaves |r|^2 = 1 + O(d^2);
// r1 is made orthogonal to the normalised r0 first.  d is accumulated from -1 by FMAs,
// so it is never rounded as 1 + d (in FP32 that would quantise it to 6e-8 steps), and
// the scaling is one FMA per entry.  The complex sums run on the paired FMAs.
DEV CA<float> as_acc(cx<float> z) { return {pk2(z.r, z.i)}; }
DEV CA<double> as_acc(cx<double> z) { return {z}; }
template <class T> DEV T norm2_minus_one(const cx<T>* r) {
    return val(ccmac(ccmac(ccmac(as_acc(mk(T(-1), T(0))), r[0], r[0]), r[1], r[1]), r[2], r[2])).r;
}
template <class T> DEV void renorm_rows(M3<T>& U) {
    const T h0 = T(-0.5) * norm2_minus_one(U.m[0]);
#pragma unroll
    for (int k = 0; k < 3; k++) U.m[0][k] = val(rmac(as_acc(U.m[0][k]), h0, U.m[0][k]));
    const cx<T> ip = val(ccmac(ccmac(ccmul(U.m[0][0], U.m[1][0]), U.m[0][1], U.m[1][1]), U.m[0][2], U.m[1][2]));
    const cx<T> mip = mk(-ip.r, -ip.i);
#pragma unroll
    for (int k = 0; k < 3; k++) U.m[1][k] = val(cmac(as_acc(U.m[1][k]), mip, U.m[0][k]));
    const T h1 = T(-0.5) * norm2_minus_one(U.m[1]);
#pragma unroll
    for (int k = 0; k < 3; k++) U.m[1][k] = val(rmac(as_acc(U.m[1][k]), h1, U.m[1][k]));
}

// Gram-Schmidt of rows 0, 1 in FP64 (row 2 is implied)
template <class T> DEV void reunit_rows(M3<T>& U) {
    double r0[6], r1[6];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        r0[2 * k] = (double)U.m[0][k].r; r0[2 * k + 1] = (double)U.m[0][k].i;
        r1[2 * k] = (double)U.m[1][k].r; r1[2 * k + 1] = (double)U.m[1][k].i;
    }
    double n0 = 0;
#pragma unroll
    for (int k = 0; k < 6; k++) n0 += r0[k] * r0[k];
    n0 = rsqrt(n0);
#pragma unroll
    for (int k = 0; k < 6; k++) r0[k] *= n0;
    // <r0, r1> = sum conj(r0_k) r1_k
    double ipr = 0, ipi = 0;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        ipr += r0[2 * k] * r1[2 * k] + r0[2 * k + 1] * r1[2 * k + 1];
        ipi += r0[2 * k] * r1[2 * k + 1] - r0[2 * k + 1] * r1[2 * k];
    }
#pragma unroll
    for (int k = 0; k < 3; k++) {
        r1[2 * k] -= ipr * r0[2 * k] - ipi * r0[2 * k + 1];
        r1[2 * k + 1] -= ipr * r0[2 * k + 1] + ipi * r0[2 * k];
    }
    double n1 = 0;
#pragma unroll
    for (int k = 0; k < 6; k++) n1 += r1[k] * r1[k];
    n1 = rsqrt(n1);
#pragma unroll
    for (int k = 0; k < 3; k++) {
        U.m[0][k] = mk((T)r0[2 * k], (T)r0[2 * k + 1]);
        U.m[1][k] = mk((T)(r1[2 * k] * n1), (T)(r1[2 * k + 1] * n1));
    }
    complete_row2(U);
}

}  // namespace glasma
