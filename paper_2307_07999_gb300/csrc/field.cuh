// Field-buffer layout and the fused kick+drift step of the boost-invariant
// Glasma leapfrog (Sec. 1 "Glasma" of arXiv:2307.07999: lattice gauge links and
// plaquettes in Milne coordinates).
//
// One field buffer holds 56 planes of n*n reals (site s = x + n*y, x fastest):
//   planes  0..11 : U_x rows 0,1 (re, im interleaved per entry)
//   planes 12..23 : U_y rows 0,1
//   planes 24..31 : E_x^a        planes 32..39 : E_y^a
//   planes 40..47 : phi^a        planes 48..55 : pi^a
// The planes come in 14 groups of four, each group interleaved per site: plane p of
// site s sits at ((p / 4) * n*n + s) * 4 + p % 4.  Four consecutive planes of a site
// are one 16-byte (FP32) or 32-byte (FP64) vector, so a link is three vector loads
// and an algebra field two, coalesced across a warp of consecutive sites and one
// sector each for a particle's scattered gather.
// Staggering: U, phi at tau_n;  E, pi at tau_{n-1/2}.
#pragma once
#include "su3.cuh"

namespace glasma {

enum { P_UX = 0, P_UY = 12, P_EX = 24, P_EY = 32, P_PHI = 40, P_PI = 48, N_PLANES = 56 };

template <class T> struct StepArgs {
    const T* src;  // state at step n
    T* dst;        // state at step n+1
    int n;
    T tb;          // plaquette-force factor: tau_n (expanding) or 1
    T tp;          // phi-sector factor:      1/tau_n (expanding) or 1
    T dtau;
    T ue;          // link drift:  dtau / tau_{n+1/2} (or dtau)
    T pe;          // phi drift:   dtau * tau_{n+1/2} (or dtau)
    int reunit;    // Gram-Schmidt the new links in FP64
};

struct TileItem { int ev, x0, y0; };

DEV size_t fidx(int p, size_t s, size_t ns) { return (((size_t)(p >> 2) * ns + s) << 2) + (p & 3); }

// Global loads of field data: through the read-only cache when the data is constant for
// the whole kernel (CG = false), at L2 (coherent) inside a persistent kernel that also
// writes the buffers it reads in later phases (CG = true).
template <bool CG, class T> DEV T ldf(const T* p) {
    if constexpr (CG) return __ldcg(p);
    else return __ldg(p);
}
template <class T> struct V4 { T v[4]; };
template <bool CG> DEV V4<float> ld4(const float* p) {
    const float4 q = CG ? __ldcg(reinterpret_cast<const float4*>(p)) : __ldg(reinterpret_cast<const float4*>(p));
    return V4<float>{{q.x, q.y, q.z, q.w}};
}
template <bool CG> DEV V4<double> ld4(const double* p) {
    const double2* v = reinterpret_cast<const double2*>(p);
    const double2 a = CG ? __ldcg(v) : __ldg(v), b = CG ? __ldcg(v + 1) : __ldg(v + 1);
    return V4<double>{{a.x, a.y, b.x, b.y}};
}
DEV void st4(float* p, float a, float b, float c, float d) { *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d); }
DEV void st4(double* p, double a, double b, double c, double d) {
    double2* v = reinterpret_cast<double2*>(p);
    v[0] = make_double2(a, b);
    v[1] = make_double2(c, d);
}
// group-aligned plane0 (a multiple of 4): rows 0,1 of a link, third row completed
template <class T, bool CG = false> DEV M3<T> load_link(const T* __restrict__ f, size_t ns, int plane0, size_t s) {
    M3<T> U;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const V4<T> q = ld4<CG>(f + fidx(plane0 + 4 * k, s, ns));
        // group k holds entries 2k and 2k+1 of rows 0,1 (row-major), re/im interleaved
        U.m[(2 * k) / 3][(2 * k) % 3] = mk(q.v[0], q.v[1]);
        U.m[(2 * k + 1) / 3][(2 * k + 1) % 3] = mk(q.v[2], q.v[3]);
    }
    complete_row2(U);
    return U;
}
template <class T> DEV void store_link(T* __restrict__ f, size_t ns, int plane0, size_t s, const M3<T>& U) {
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const cx<T> a = U.m[(2 * k) / 3][(2 * k) % 3], b = U.m[(2 * k + 1) / 3][(2 * k + 1) % 3];
        st4(f + fidx(plane0 + 4 * k, s, ns), a.r, a.i, b.r, b.i);
    }
}
template <class T, bool CG = false> DEV Al<T> load_alg(const T* __restrict__ f, size_t ns, int plane0, size_t s) {
    Al<T> x;
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const V4<T> q = ld4<CG>(f + fidx(plane0 + 4 * k, s, ns));
#pragma unroll
        for (int j = 0; j < 4; j++) x.a[4 * k + j] = q.v[j];
    }
    return x;
}
template <class T> DEV void store_alg(T* __restrict__ f, size_t ns, int plane0, size_t s, const Al<T>& x) {
#pragma unroll
    for (int k = 0; k < 2; k++) st4(f + fidx(plane0 + 4 * k, s, ns), x.a[4 * k], x.a[4 * k + 1], x.a[4 * k + 2], x.a[4 * k + 3]);
}
DEV int wrapi(int v, int n) { v %= n; return v < 0 ? v + n : v; }

template <class T, int TX, int TY> struct Tile {
    static constexpr int HX = TX + 2, HY = TY + 2, HS = HX * HY;
    static constexpr int FX = TX + 1, FY = TY + 1, FS = FX * FY;
    static constexpr size_t smem = sizeof(T) * (size_t)(2 * 18 * HS + 8 * HS + 8 * FS);
};

template <class T, int HS> DEV M3<T> sm_link(const T* sU, int d, int h) {
    M3<T> U;
    const T* b = sU + d * 18 * HS + h;
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int c = 0; c < 3; c++) U.m[r][c] = mk(b[(2 * (3 * r + c)) * HS], b[(2 * (3 * r + c) + 1) * HS]);
    return U;
}
template <class T, int S> DEV Al<T> sm_alg(const T* s, int h) {
    Al<T> x;
#pragma unroll
    for (int a = 0; a < 8; a++) x.a[a] = s[a * S + h];
    return x;
}

// One tile [x0, x0+TX) x [y0, y0+TY) of one step: kick at tau_n, drift with tau_{n+1/2}.
template <class T, int TX, int TY, bool CG = false>
DEV void field_tile(const StepArgs<T>& A, int x0, int y0, unsigned char* smem_raw) {
    using G = Tile<T, TX, TY>;
    constexpr int HX = G::HX, HS = G::HS, FX = G::FX, FS = G::FS;
    T* sU = reinterpret_cast<T*>(smem_raw);  // [2][18][HS]
    T* sP = sU + 2 * 18 * HS;                // [8][HS]  phi
    T* sF = sP + 8 * HS;                     // [8][FS]  ImTL of the plaquette
    const int n = A.n;
    const size_t ns = (size_t)n * n;
    const int tid = threadIdx.y * TX + threadIdx.x;
    const T* __restrict__ src = A.src;

    // own E, pi: issue the loads early
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    const bool active = (x < n) && (y < n);
    const size_t s = active ? (size_t)x + (size_t)n * y : 0;
    Al<T> Ex = load_alg<T, CG>(src, ns, P_EX, s), Ey = load_alg<T, CG>(src, ns, P_EY, s), pi = load_alg<T, CG>(src, ns, P_PI, s);

    // phase 1: links (completed to 3 rows) and phi of the tile plus a one-site halo
    for (int h = tid; h < HS; h += TX * TY) {
        const int hx = h % HX, hy = h / HX;
        const size_t g = (size_t)wrapi(x0 - 1 + hx, n) + (size_t)n * wrapi(y0 - 1 + hy, n);
#pragma unroll
        for (int d = 0; d < 2; d++) {
            const M3<T> U = load_link<T, CG>(src, ns, d == 0 ? P_UX : P_UY, g);
            T* b = sU + d * 18 * HS + h;
#pragma unroll
            for (int r = 0; r < 3; r++)
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    b[(2 * (3 * r + c)) * HS] = U.m[r][c].r;
                    b[(2 * (3 * r + c) + 1) * HS] = U.m[r][c].i;
                }
        }
        const Al<T> ph = load_alg<T, CG>(src, ns, P_PHI, g);
#pragma unroll
        for (int a = 0; a < 8; a++) sP[a * HS + h] = ph.a[a];
    }
    __syncthreads();

    // phase 2: ImTL P(x) for x in [x0-1, x0+TX) x [y0-1, y0+TY)
    for (int i = tid; i < FS; i += TX * TY) {
        const int fx = i % FX, fy = i / FX;
        const int h = fy * HX + fx;
        const M3<T> a1 = mul(sm_link<T, HS>(sU, 0, h), sm_link<T, HS>(sU, 1, h + 1));
        const M3<T> b1 = mul(sm_link<T, HS>(sU, 1, h), sm_link<T, HS>(sU, 0, h + HX));
        const Al<T> F = im_tl(mul_nd(a1, b1));
#pragma unroll
        for (int a = 0; a < 8; a++) sF[a * FS + i] = F.a[a];
    }
    __syncthreads();
    if (!active) return;

    // phase 3: kick and drift of the own site
    const int h = (threadIdx.y + 1) * HX + threadIdx.x + 1;
    const int f = (threadIdx.y + 1) * FX + threadIdx.x + 1;
    const Al<T> phi = sm_alg<T, HS>(sP, h);
    const M3<T> ux = sm_link<T, HS>(sU, 0, h), uy = sm_link<T, HS>(sU, 1, h);
    const M3<T> uxm = sm_link<T, HS>(sU, 0, h - 1), uym = sm_link<T, HS>(sU, 1, h - HX);
    const T dt = A.dtau, tb = A.tb, tp = A.tp;

    const Al<T> psx = conj_alg(ux, sm_alg<T, HS>(sP, h + 1));
    const Al<T> psy = conj_alg(uy, sm_alg<T, HS>(sP, h + HX));
    {
        const Al<T> chx = transport_alg(uxm, sm_alg<T, HS>(sP, h - 1));
        const Al<T> chy = transport_alg(uym, sm_alg<T, HS>(sP, h - HX));
#pragma unroll
        for (int a = 0; a < 8; a++)
            pi.a[a] += dt * tp * (psx.a[a] + chx.a[a] + psy.a[a] + chy.a[a] - T(4) * phi.a[a]);
    }
    const Al<T> F0 = sm_alg<T, FS>(sF, f);
    {
        const Al<T> cm = icomm(phi, psx);
        const Al<T> t1 = transport_alg(uym, sm_alg<T, FS>(sF, f - FX));
#pragma unroll
        for (int a = 0; a < 8; a++) Ex.a[a] += dt * (tb * (t1.a[a] - F0.a[a]) - tp * cm.a[a]);
    }
    {
        const Al<T> cm = icomm(phi, psy);
        const Al<T> t2 = transport_alg(uxm, sm_alg<T, FS>(sF, f - 1));
#pragma unroll
        for (int a = 0; a < 8; a++) Ey.a[a] += dt * (tb * (F0.a[a] - t2.a[a]) - tp * cm.a[a]);
    }
    T* __restrict__ dst = A.dst;
    store_alg(dst, ns, P_EX, s, Ex);
    store_alg(dst, ns, P_EY, s, Ey);
    store_alg(dst, ns, P_PI, s, pi);
    Al<T> phin;
#pragma unroll
    for (int a = 0; a < 8; a++) phin.a[a] = phi.a[a] + A.pe * pi.a[a];
    store_alg(dst, ns, P_PHI, s, phin);
    // drift of the links: U <- exp(i ue E) U
#pragma unroll
    for (int d = 0; d < 2; d++) {
        Al<T> e = d == 0 ? Ex : Ey;
#pragma unroll
        for (int a = 0; a < 8; a++) e.a[a] *= A.ue;
        const M3<T> W = expi(herm(e));
        const M3<T>& U = d == 0 ? ux : uy;
        M3<T> V;
#pragma unroll
        for (int r = 0; r < 2; r++)
#pragma unroll
            for (int c = 0; c < 3; c++) {
                cx<T> v = W.m[r][0] * U.m[0][c];
                fma_(v, W.m[r][1], U.m[1][c]);
                fma_(v, W.m[r][2], U.m[2][c]);
                V.m[r][c] = v;
            }
        if (A.reunit) reunit_rows(V);
        store_link(dst, ns, d == 0 ? P_UX : P_UY, s, V);
    }
}

}  // namespace glasma
