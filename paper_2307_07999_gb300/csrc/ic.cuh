// MV-model initial conditions on the device (Sec. 1 "Glasma", Eq. 1 of
// arXiv:2307.07999; the lattice matching at tau = 0+ is the standard
// boost-invariant one, the paper defers it to its companion paper).
//   charges   rho^a_{A,n}(x) ~ N(0, (g^2 mu a)^2 / Ns)    (Philox4x32-10 + Box-Muller)
//   Poisson   Lambda = (k~^2 + m^2)^-1 rho, zero mode 0  (cuFFT Z2Z, k~^2 = sum 4 sin^2(pi k/N))
//   Wilson    V_A <- exp(-i Lambda_{A,n}) V_A, sheet 1 first
//   links     U^(A)_i(x) = V_A(x) V_A(x+i)^dag
//   matching  Im Tr[t^a (U1 + U2)(1 + U^dag)] = 0, Newton in U <- exp(i d.t) U, step
//             halving, start U1 U2 (restart from 1 if it stalls); the warm start
//             exp(i (d_series + d_net).t) U1 U2 adds a third-order series and a
//             learned correction (mlp.cu)
//   pi(0)     -(i/4) sum_i {[(U-1)(U2^dag - U1^dag) - h.c.](x) + [(U^dag-1)(U2 - U1) - h.c.](x-i)}
// All initial-condition arithmetic is FP64, whatever the evolution precision.
#pragma once
#include "field.cuh"

namespace glasma {

// ---------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror, Shaw, SC'11: 10 rounds of two 32x32->64 multiplies and a
// key-dependent xor mix, Weyl key schedule between rounds.
DEV uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; r++) {
        if (r) { k.x += 0x9E3779B9u; k.y += 0xBB67AE85u; }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}
DEV double u01(uint32_t r) { return ((double)r + 0.5) * 2.3283064365386962890625e-10; }
DEV void box_muller(uint32_t a, uint32_t b, double& g0, double& g1) {
    const double rad = sqrt(-2.0 * log(u01(a)));
    double s, c;
    sincospi(2.0 * u01(b), &s, &c);
    g0 = rad * c;
    g1 = rad * s;
}
DEV uint2 seed_key(uint64_t seed) { return make_uint2((uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)); }

// ---------------------------------------------------------------- generators as matrices
DEV M3<double> gen(int a) {
    M3<double> t;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) t.m[i][j] = mk(0.0, 0.0);
    const double h = 0.5, s8 = 0.28867513459481288225;  // 1/(2 sqrt 3)
    switch (a) {
        case 0: t.m[0][1] = mk(h, 0.0); t.m[1][0] = mk(h, 0.0); break;
        case 1: t.m[0][1] = mk(0.0, -h); t.m[1][0] = mk(0.0, h); break;
        case 2: t.m[0][0] = mk(h, 0.0); t.m[1][1] = mk(-h, 0.0); break;
        case 3: t.m[0][2] = mk(h, 0.0); t.m[2][0] = mk(h, 0.0); break;
        case 4: t.m[0][2] = mk(0.0, -h); t.m[2][0] = mk(0.0, h); break;
        case 5: t.m[1][2] = mk(h, 0.0); t.m[2][1] = mk(h, 0.0); break;
        case 6: t.m[1][2] = mk(0.0, -h); t.m[2][1] = mk(0.0, h); break;
        default: t.m[0][0] = mk(s8, 0.0); t.m[1][1] = mk(s8, 0.0); t.m[2][2] = mk(-2.0 * s8, 0.0); break;
    }
    return t;
}
// components 2 Re Tr(t^a Y) of a general matrix (those of its Hermitian part)
DEV Al<double> re_comp(const M3<double>& M) {
    Al<double> x;
    x.a[0] = M.m[0][1].r + M.m[1][0].r;
    x.a[1] = M.m[1][0].i - M.m[0][1].i;
    x.a[2] = M.m[0][0].r - M.m[1][1].r;
    x.a[3] = M.m[0][2].r + M.m[2][0].r;
    x.a[4] = M.m[2][0].i - M.m[0][2].i;
    x.a[5] = M.m[1][2].r + M.m[2][1].r;
    x.a[6] = M.m[2][1].i - M.m[1][2].i;
    x.a[7] = (M.m[0][0].r + M.m[1][1].r - 2.0 * M.m[2][2].r) * 0.57735026918962576451;
    return x;
}
DEV M3<double> ident() {
    M3<double> I;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) I.m[i][j] = mk(i == j ? 1.0 : 0.0, 0.0);
    return I;
}
DEV M3<double> dag(const M3<double>& A) {
    M3<double> B;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) B.m[i][j] = cj(A.m[j][i]);
    return B;
}
DEV M3<double> addm(const M3<double>& A, const M3<double>& B, double sb = 1.0) {
    M3<double> C;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) C.m[i][j] = mk(A.m[i][j].r + sb * B.m[i][j].r, A.m[i][j].i + sb * B.m[i][j].i);
    return C;
}

// full 3x3 link AoS in scratch: 18 doubles per link
DEV M3<double> ld18(const double* p) {
    M3<double> U;
#pragma unroll
    for (int k = 0; k < 9; k++) U.m[k / 3][k % 3] = mk(p[2 * k], p[2 * k + 1]);
    return U;
}
DEV void st18(double* p, const M3<double>& U) {
#pragma unroll
    for (int k = 0; k < 9; k++) { p[2 * k] = U.m[k / 3][k % 3].r; p[2 * k + 1] = U.m[k / 3][k % 3].i; }
}

// residual r^a = Im Tr[t^a S (1 + U^dag)] = (1/2) ImTL(S (1 + U^dag))^a
DEV Al<double> ic_residual(const M3<double>& S, const M3<double>& U) {
    const M3<double> M = mul(S, addm(ident(), dag(U)));
    Al<double> r = im_tl(M);
#pragma unroll
    for (int a = 0; a < 8; a++) r.a[a] *= 0.5;
    return r;
}
DEV double nrm8(const Al<double>& r) {
    double s = 0;
#pragma unroll
    for (int a = 0; a < 8; a++) s += r.a[a] * r.a[a];
    return sqrt(s);
}
// J d = b (8x8, partial pivoting); returns false if singular
DEV bool solve8(double J[8][8], double b[8], double d[8]) {
    for (int c = 0; c < 8; c++) {
        int p = c;
        for (int i = c + 1; i < 8; i++)
            if (fabs(J[i][c]) > fabs(J[p][c])) p = i;
        if (fabs(J[p][c]) < 1e-300) return false;
        if (p != c) {
            for (int j = 0; j < 8; j++) { const double t = J[c][j]; J[c][j] = J[p][j]; J[p][j] = t; }
            const double t = b[c]; b[c] = b[p]; b[p] = t;
        }
        for (int i = c + 1; i < 8; i++) {
            const double f = J[i][c] / J[c][c];
            for (int j = c; j < 8; j++) J[i][j] -= f * J[c][j];
            b[i] -= f * b[c];
        }
    }
    for (int i = 7; i >= 0; i--) {
        double s = b[i];
        for (int j = i + 1; j < 8; j++) s -= J[i][j] * d[j];
        d[i] = s / J[i][i];
    }
    return true;
}
// Small-field series of the solution's offset from U1 U2: U = exp(i d.t) U1 U2 with
//   d = -c/2 - (3/8) i[a1, c] - (1/8) i[a2, c] + O(a^4),  a_k = im_tl(U_k), c = i[a1, a2]
// (obtained by expanding the matching condition order by order in the link fields).
template <class T> struct IcSeries {
    Al<T> a1, a2, c, cubic;  // cubic = d + c/2
};
template <class T> DEV IcSeries<T> ic_series(const M3<T>& U1, const M3<T>& U2) {
    IcSeries<T> q;
    q.a1 = im_tl(U1);
    q.a2 = im_tl(U2);
    q.c = icomm(q.a1, q.a2);
    const Al<T> c1 = icomm(q.a1, q.c), c2 = icomm(q.a2, q.c);
#pragma unroll
    for (int a = 0; a < 8; a++) q.cubic.a[a] = T(-0.375) * c1.a[a] - T(0.125) * c2.a[a];
    return q;
}
template <class T> DEV Al<T> series_offset(const IcSeries<T>& q) {
    Al<T> d;
#pragma unroll
    for (int a = 0; a < 8; a++) d.a[a] = T(-0.5) * q.c.a[a] + q.cubic.a[a];
    return d;
}
// FP32 copy of an FP64 matrix (warm-start inputs need no more)
DEV M3<float> to_f32(const M3<double>& A) {
    M3<float> B;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) B.m[i][j] = mk((float)A.m[i][j].r, (float)A.m[i][j].i);
    return B;
}
// One Newton step with step halving on U (residual norm rn at U on entry).  Returns
// false when the Jacobian is singular (U unchanged); otherwise U and rn hold the new
// iterate and *stalled tells whether no halving reduced the residual.
DEV bool newton_step(const M3<double>& S, M3<double>& U, Al<double>& r, double& rn, bool* stalled) {
    // J_ab = -Re Tr[t^a (S U^dag) t^b] = -(1/2) re_comp(S U^dag t^b)^a
    const M3<double> SU = mul_nd(S, U);
    double J[8][8], b[8], d[8];
    for (int bb = 0; bb < 8; bb++) {
        const Al<double> col = re_comp(mul(SU, gen(bb)));
#pragma unroll
        for (int a = 0; a < 8; a++) J[a][bb] = -0.5 * col.a[a];
    }
#pragma unroll
    for (int a = 0; a < 8; a++) b[a] = -r.a[a];
    if (!solve8(J, b, d)) return false;
    double lam = 1.0, rnn = 0.0;
    M3<double> Un = U;
    Al<double> rnew = r;
    for (int h = 0; h < 12; h++) {
        Al<double> dx;
#pragma unroll
        for (int a = 0; a < 8; a++) dx.a[a] = lam * d[a];
        Un = mul(expi(herm(dx)), U);
        rnew = ic_residual(S, Un);
        rnn = nrm8(rnew);
        if (rnn < rn) break;
        lam *= 0.5;
    }
    *stalled = !(rnn < rn);
    U = Un;
    r = rnew;
    rn = rnn;
    return true;
}
// Newton with step halving from the given U; returns iterations or -1
DEV int newton_link(const M3<double>& U1, const M3<double>& U2, M3<double>& U, double tol, int max_iter,
                    double& res) {
    const M3<double> S = addm(U1, U2);
    Al<double> r = ic_residual(S, U);
    double rn = nrm8(r);
    int it = 0;
    while (rn > tol && it < max_iter) {
        bool stalled = false;
        if (!newton_step(S, U, r, rn, &stalled)) break;
        it++;
        if (stalled) break;
    }
    res = rn;
    return rn <= tol ? it : -1;
}

}  // namespace glasma
