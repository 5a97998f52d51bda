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
    U.m[2][0] = cj(a[1] * b[2] - a[2] * b[1]);
    U.m[2][1] = cj(a[2] * b[0] - a[0] * b[2]);
    U.m[2][2] = cj(a[0] * b[1] - a[1] * b[0]);
}
// C = A B
template <class T> DEV M3<T> mul(const M3<T>& A, const M3<T>& B) {
    M3<T> C;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            cx<T> s = A.m[i][0] * B.m[0][j];
            fma_(s, A.m[i][1], B.m[1][j]);
            fma_(s, A.m[i][2], B.m[2][j]);
            C.m[i][j] = s;
        }
    return C;
}
// C = A B^dag
template <class T> DEV M3<T> mul_nd(const M3<T>& A, const M3<T>& B) {
    M3<T> C;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            cx<T> s = mulc(A.m[i][0], B.m[j][0]);
            fmac_(s, A.m[i][1], B.m[j][1]);
            fmac_(s, A.m[i][2], B.m[j][2]);
            C.m[i][j] = s;
        }
    return C;
}
// ImTL(A B^dag) without forming the real parts of the diagonal
template <class T> DEV Al<T> im_tl_nd(const M3<T>& A, const M3<T>& B) {
    return im_tl(mul_nd(A, B));
}

// U^dag X U for Hermitian X (result Hermitian; only diagonal + upper computed)
template <class T> DEV H3<T> transport(const M3<T>& U, const H3<T>& X) {
    // W = X U
    M3<T> W;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            cx<T> s = mk(T(0), T(0));
#pragma unroll
            for (int k = 0; k < 3; k++) fma_(s, hget(X, i, k), U.m[k][j]);
            W.m[i][j] = s;
        }
    // R = U^dag W, R_ij = sum_k conj(U_ki) W_kj
    H3<T> R;
    cx<T> r;
#define GL_RIJ(i, j)                                        \
    r = mk(T(0), T(0));                                     \
    fmca_(r, U.m[0][i], W.m[0][j]);                         \
    fmca_(r, U.m[1][i], W.m[1][j]);                         \
    fmca_(r, U.m[2][i], W.m[2][j]);
    GL_RIJ(0, 0) R.d0 = r.r;
    GL_RIJ(1, 1) R.d1 = r.r;
    GL_RIJ(2, 2) R.d2 = r.r;
    GL_RIJ(0, 1) R.u01 = r;
    GL_RIJ(0, 2) R.u02 = r;
    GL_RIJ(1, 2) R.u12 = r;
#undef GL_RIJ
    return R;
}
// U X U^dag for Hermitian X
template <class T> DEV H3<T> conj_by(const M3<T>& U, const H3<T>& X) {
    // W = U X
    M3<T> W;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            cx<T> s = mk(T(0), T(0));
#pragma unroll
            for (int k = 0; k < 3; k++) fma_(s, U.m[i][k], hget(X, k, j));
            W.m[i][j] = s;
        }
    // R_ij = sum_k W_ik conj(U_jk)
    H3<T> R;
    cx<T> r;
#define GL_RIJ(i, j)                                        \
    r = mk(T(0), T(0));                                     \
    fmac_(r, W.m[i][0], U.m[j][0]);                         \
    fmac_(r, W.m[i][1], U.m[j][1]);                         \
    fmac_(r, W.m[i][2], U.m[j][2]);
    GL_RIJ(0, 0) R.d0 = r.r;
    GL_RIJ(1, 1) R.d1 = r.r;
    GL_RIJ(2, 2) R.d2 = r.r;
    GL_RIJ(0, 1) R.u01 = r;
    GL_RIJ(0, 2) R.u02 = r;
    GL_RIJ(1, 2) R.u12 = r;
#undef GL_RIJ
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

template <class T> struct ExpTerms { static constexpr int K = 16; };
template <> struct ExpTerms<float> { static constexpr int K = 9; };

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
            cx<T> w = f1 * hget(X, i, j);
            fma_(w, f2, hget(X2, i, j));
            if (i == j) w = w + f0;
            W.m[i][j] = w;
        }
    return W;
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
