// Field-buffer layout and the fused kick+drift step of the boost-invariant
// Glasma leapfrog (Sec. 1 "Glasma" of arXiv:2307.07999: lattice gauge links and
// plaquettes in Milne coordinates).
//
// One field buffer holds 64 planes of n*n reals (site s = x + n*y, x fastest):
//   planes  0..11 : U_x rows 0,1 (re, im interleaved per entry)
//   planes 12..23 : U_y rows 0,1
//   planes 24..31 : E_x^a        planes 32..39 : E_y^a
//   planes 40..47 : phi^a        planes 48..55 : pi^a
//   planes 56..63 : F^a = ImTL of the plaquette based at the site, of the links of this
//                   buffer: not state; written by the one-event field step that reads the
//                   buffer (it forms them anyway for the staples) for the push of that step
// The planes come in 8 groups of eight, each group interleaved per site: plane p of
// site s sits at ((p / 8) * n*n + s) * 8 + p % 8.  A group of one site is one 32-byte
// sector in FP32, loaded as two 16-byte vectors: a warp of consecutive sites reads
// contiguous memory, and a particle's scattered gather touches few sectors (both
// links of a cell: three; E_x and E_y: two; phi, pi: one each).
// Staggering: U, phi at tau_n;  E, pi at tau_{n-1/2}.
#pragma once
#include "su3.cuh"

namespace glasma {

enum { P_UX = 0, P_UY = 12, P_EX = 24, P_EY = 32, P_PHI = 40, P_PI = 48, P_F = 56, N_PLANES = 64 };

template <class T> struct StepArgs {
    const T* src;  // state at step n
    T* dst;        // state at step n+1
    int n;
    T tb;          // plaquette-force factor: tau_n (expanding) or 1
    T tp;          // phi-sector factor:      1/tau_n (expanding) or 1
    T dtau;
    T ue;          // link drift:  dtau / tau_{n+1/2} (or dtau)
    T pe;          // phi drift:   dtau * tau_{n+1/2} (or dtau)
    int reunit;    // re-projection of the new links: 1 FP64 Gram-Schmidt, 2 FP32 renormalisation, 0 none
    T* plaq;       // the source buffer again, whose group P_F receives ImTL of each site's
                   // plaquette (kernels compiled with PLAQ: the one-event step)
    // gather records (kernels compiled with REC only): for every cell whose occupancy
    // stamp equals `epoch` (every cell if all_rec), the pieces of the site-centred fields
    // that the push of this step gathers there (layout below)
    T* rec;
    const int* occ;
    int epoch, all_rec;
};

// Gather record of a cell c for the push of step n (8-real groups; REC_STRIDE groups per
// record, so that in FP32 a record is five whole 128-byte lines).  Written by the field
// step of step n, which computes each piece anyway.  Each writer fills whole lines (the
// unused groups are written as zeros), so the records reach DRAM as full lines:
//   lines 0-2, the owner of c:
//     R_EX, R_EY, R_PI  time-centred E_x(c), E_y(c), pi(c): (X_{n-1/2} + X_{n+1/2}) / 2
//     R_PHI             phi_n(c)
//     R_PSX, R_CHX      U_x(c) phi(c+x) U_x(c)^dag and U_x(c-x)^dag phi(c-x) U_x(c-x)
//     R_PSY, R_CHY      the same along y
//     R_F0              ImTL of the plaquette based at c
//     R_T1, R_T2        ImTL of the plaquettes at c-y and c-x carried to c by U_y(c-y), U_x(c-x)
//                       (the clover leaves (-y,+x) and (+y,-x) of c)
//   line 3, the owner of c-x:  R_EXL time-centred E_x(c-x), R_T1L its R_T1, R_UXL (2 groups)
//                              U_x(c-x) rows 0, 1
//   line 4, the owner of c-y:  R_EYB time-centred E_y(c-y), R_UYB (2 groups) U_y(c-y) rows 0, 1
// so that Q.E_x(c) = (Q.E_x(c) + Q'.E_x(c-x)) / 2 with Q' = U_x(c-x) Q U_x(c-x)^dag, and the
// fourth clover leaf (-x,-y) of c contracts as Q'.R_T1L.
enum {
    R_EX = 0, R_EY, R_PI, R_PHI, R_PSX, R_CHX, R_PSY, R_CHY, R_F0, R_T1, R_T2, R_PAD0,
    R_EXL = 12, R_T1L, R_UXL,
    R_EYB = 16, R_UYB, R_PAD1 = 19, REC_STRIDE = 20
};

struct TileItem { int ev, x0, y0; };

DEV size_t fidx(int p, size_t s, size_t ns) { return (((size_t)(p >> 3) * ns + s) << 3) + (p & 7); }

// Global loads of field data: through the read-only cache when the data is constant for
// the whole kernel (CG = false), at L2 (coherent) inside a persistent kernel that also
// writes the buffers it reads in later phases (CG = true).
template <bool CG, class T> DEV T ldf(const T* p) {
    if constexpr (CG) return __ldcg(p);
    else return __ldg(p);
}
template <class T> struct V4 { T v[4]; };
template <class T> struct V8 { T v[8]; };
template <bool CG> DEV V4<float> ld4(const float* p) {
    const float4 q = CG ? __ldcg(reinterpret_cast<const float4*>(p)) : __ldg(reinterpret_cast<const float4*>(p));
    return V4<float>{{q.x, q.y, q.z, q.w}};
}
template <bool CG> DEV V4<double> ld4(const double* p) {
    const double2* v = reinterpret_cast<const double2*>(p);
    const double2 a = CG ? __ldcg(v) : __ldg(v), b = CG ? __ldcg(v + 1) : __ldg(v + 1);
    return V4<double>{{a.x, a.y, b.x, b.y}};
}
// one plane group of a site: a 32-byte load in FP32 (sm_100 family 256-bit access;
// the address is 32-byte aligned), two in FP64.  The non-coherent form is a plain
// asm (it may be scheduled freely: the data is constant for the kernel); the
// coherent form is volatile so that it stays on its side of the persistent
// kernel's grid barriers.
template <bool CG> DEV V8<float> ld8(const float* p) {
    V8<float> r;
    if constexpr (CG)
        asm volatile("ld.global.cg.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3]), "=f"(r.v[4]), "=f"(r.v[5]),
                       "=f"(r.v[6]), "=f"(r.v[7])
                     : "l"(p)
                     : "memory");
    else
        asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
            : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3]), "=f"(r.v[4]), "=f"(r.v[5]), "=f"(r.v[6]),
              "=f"(r.v[7])
            : "l"(p));
    return r;
}
template <bool CG> DEV V8<double> ld8(const double* p) {
    const V4<double> a = ld4<CG>(p), b = ld4<CG>(p + 4);
    return V8<double>{{a.v[0], a.v[1], a.v[2], a.v[3], b.v[0], b.v[1], b.v[2], b.v[3]}};
}
DEV void st4(float* p, float a, float b, float c, float d) { *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d); }
DEV void st4(double* p, double a, double b, double c, double d) {
    double2* v = reinterpret_cast<double2*>(p);
    v[0] = make_double2(a, b);
    v[1] = make_double2(c, d);
}
DEV void st8(float* p, const V8<float>& x) {
    asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(x.v[0]), "f"(x.v[1]), "f"(x.v[2]),
                 "f"(x.v[3]), "f"(x.v[4]), "f"(x.v[5]), "f"(x.v[6]), "f"(x.v[7])
                 : "memory");
}
DEV void st8(double* p, const V8<double>& x) {
    st4(p, x.v[0], x.v[1], x.v[2], x.v[3]);
    st4(p + 4, x.v[4], x.v[5], x.v[6], x.v[7]);
}
// entry e = 0..5 of rows 0,1 of a link (row-major) from the 12 reals of its planes
template <class T> DEV void put_entry(M3<T>& U, int e, T re, T im) { U.m[e / 3][e % 3] = mk(re, im); }

// plane0 a multiple of 4 (planes plane0..plane0+3 are one aligned 4-vector): rows 0,1 of a
// link, third row completed
template <class T, bool CG = false> DEV M3<T> load_link(const T* __restrict__ f, size_t ns, int plane0, size_t s) {
    M3<T> U;
    if (plane0 == P_UX) {  // planes 0..7 (group 0), 8..11 (first half of group 1)
        const V8<T> a = ld8<CG>(f + fidx(0, s, ns));
        const V4<T> b = ld4<CG>(f + fidx(8, s, ns));
#pragma unroll
        for (int e = 0; e < 4; e++) put_entry(U, e, a.v[2 * e], a.v[2 * e + 1]);
        put_entry(U, 4, b.v[0], b.v[1]);
        put_entry(U, 5, b.v[2], b.v[3]);
    } else {  // planes 12..15 (second half of group 1), 16..23 (group 2)
        const V4<T> a = ld4<CG>(f + fidx(12, s, ns));
        const V8<T> b = ld8<CG>(f + fidx(16, s, ns));
        put_entry(U, 0, a.v[0], a.v[1]);
        put_entry(U, 1, a.v[2], a.v[3]);
#pragma unroll
        for (int e = 0; e < 4; e++) put_entry(U, 2 + e, b.v[2 * e], b.v[2 * e + 1]);
    }
    complete_row2(U);
    return U;
}
// both links of a site from its three link groups (planes 0-7, 8-15, 16-23)
template <class T> DEV void links_from_groups(const V8<T>& a, const V8<T>& b, const V8<T>& c, M3<T>& ux, M3<T>& uy) {
#pragma unroll
    for (int e = 0; e < 4; e++) put_entry(ux, e, a.v[2 * e], a.v[2 * e + 1]);
    put_entry(ux, 4, b.v[0], b.v[1]);
    put_entry(ux, 5, b.v[2], b.v[3]);
    put_entry(uy, 0, b.v[4], b.v[5]);
    put_entry(uy, 1, b.v[6], b.v[7]);
#pragma unroll
    for (int e = 0; e < 4; e++) put_entry(uy, 2 + e, c.v[2 * e], c.v[2 * e + 1]);
    complete_row2(ux);
    complete_row2(uy);
}
template <class T, bool CG = false> DEV void load_links(const T* __restrict__ f, size_t ns, size_t s, M3<T>& ux, M3<T>& uy) {
    links_from_groups(ld8<CG>(f + fidx(0, s, ns)), ld8<CG>(f + fidx(8, s, ns)), ld8<CG>(f + fidx(16, s, ns)), ux, uy);
}
template <class T> DEV void store_links(T* __restrict__ f, size_t ns, size_t s, const M3<T>& ux, const M3<T>& uy) {
    V8<T> a, b, c;
#pragma unroll
    for (int e = 0; e < 4; e++) {
        a.v[2 * e] = ux.m[e / 3][e % 3].r;
        a.v[2 * e + 1] = ux.m[e / 3][e % 3].i;
        c.v[2 * e] = uy.m[(e + 2) / 3][(e + 2) % 3].r;
        c.v[2 * e + 1] = uy.m[(e + 2) / 3][(e + 2) % 3].i;
    }
    b.v[0] = ux.m[1][1].r; b.v[1] = ux.m[1][1].i; b.v[2] = ux.m[1][2].r; b.v[3] = ux.m[1][2].i;
    b.v[4] = uy.m[0][0].r; b.v[5] = uy.m[0][0].i; b.v[6] = uy.m[0][1].r; b.v[7] = uy.m[0][1].i;
    st8(f + fidx(0, s, ns), a);
    st8(f + fidx(8, s, ns), b);
    st8(f + fidx(16, s, ns), c);
}
template <class T> DEV void store_link(T* __restrict__ f, size_t ns, int plane0, size_t s, const M3<T>& U) {
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const cx<T> a = U.m[(2 * k) / 3][(2 * k) % 3], b = U.m[(2 * k + 1) / 3][(2 * k + 1) % 3];
        st4(f + fidx(plane0 + 4 * k, s, ns), a.r, a.i, b.r, b.i);
    }
}
// plane0 a multiple of 8 (one group)
template <class T, bool CG = false> DEV Al<T> load_alg(const T* __restrict__ f, size_t ns, int plane0, size_t s) {
    const V8<T> q = ld8<CG>(f + fidx(plane0, s, ns));
    Al<T> x;
#pragma unroll
    for (int a = 0; a < 8; a++) x.a[a] = q.v[a];
    return x;
}
template <class T> DEV void store_alg(T* __restrict__ f, size_t ns, int plane0, size_t s, const Al<T>& x) {
    V8<T> q;
#pragma unroll
    for (int a = 0; a < 8; a++) q.v[a] = x.a[a];
    st8(f + fidx(plane0, s, ns), q);
}
DEV int wrapi(int v, int n) { v %= n; return v < 0 ? v + n : v; }

// Record tile staging of the field step: per site, a link as 20 reals (its 9 complex
// entries and two of padding) and an algebra field as 12 reals (8 and four of padding),
// moved as 16-byte vectors.  Record strides of 20 and 12 words put the eight threads
// of a quarter warp on distinct banks.
constexpr int REC_L = 20, REC_A = 12;
template <class T, int TX, int TY> struct RecTile {
    static constexpr int HX = TX + 2, HY = TY + 2, HS = HX * HY;
    static constexpr int FX = TX + 1, FY = TY + 1, FS = FX * FY;
    static constexpr size_t smem = sizeof(T) * (size_t)(2 * REC_L * HS + REC_A * HS + REC_A * FS);
};
DEV void lds_v(const float* p, float* o) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
DEV void lds_v(const double* p, double* o) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    o[0] = v.x; o[1] = v.y;
}
DEV void sts_v(float* p, const float* o) { *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]); }
DEV void sts_v(double* p, const double* o) { *reinterpret_cast<double2*>(p) = make_double2(o[0], o[1]); }
template <class T> DEV M3<T> rec_link(const T* sU, int h) {
    constexpr int NV = 16 / sizeof(T);
    T b[REC_L];
#pragma unroll
    for (int k = 0; k < REC_L; k += NV) lds_v(sU + h * REC_L + k, b + k);
    M3<T> U;
#pragma unroll
    for (int e = 0; e < 9; e++) U.m[e / 3][e % 3] = mk(b[2 * e], b[2 * e + 1]);
    return U;
}
template <class T> DEV void rec_put_link(T* sU, int h, const M3<T>& U) {
    constexpr int NV = 16 / sizeof(T);
    T b[REC_L];
#pragma unroll
    for (int e = 0; e < 9; e++) { b[2 * e] = U.m[e / 3][e % 3].r; b[2 * e + 1] = U.m[e / 3][e % 3].i; }
    b[18] = T(0);
    b[19] = T(0);
#pragma unroll
    for (int k = 0; k < REC_L; k += NV) sts_v(sU + h * REC_L + k, b + k);
}
template <class T> DEV Al<T> rec_alg(const T* s, int h) {
    constexpr int NV = 16 / sizeof(T);
    Al<T> x;
#pragma unroll
    for (int k = 0; k < 8; k += NV) lds_v(s + h * REC_A + k, x.a + k);
    return x;
}
template <class T> DEV void rec_put_alg(T* s, int h, const Al<T>& x) {
    constexpr int NV = 16 / sizeof(T);
#pragma unroll
    for (int k = 0; k < 8; k += NV) sts_v(s + h * REC_A + k, x.a + k);
}

template <class T> DEV T* rec_at(T* rec, size_t cell, int slot) {
    return rec + (cell * REC_STRIDE + (size_t)slot) * 8;
}
// Record stores: plain C++ 256-bit stores under a condition, which the compiler turns into
// predicated stores and schedules with the step's arithmetic (inline-asm stores are kept in
// program order, which holds their operands live and raised the step's local-memory use).
DEV void st8_if(bool p, float* a, const V8<float>& v) {
    ulonglong4_32a w;
    w.x = ((unsigned long long)__float_as_uint(v.v[1]) << 32) | __float_as_uint(v.v[0]);
    w.y = ((unsigned long long)__float_as_uint(v.v[3]) << 32) | __float_as_uint(v.v[2]);
    w.z = ((unsigned long long)__float_as_uint(v.v[5]) << 32) | __float_as_uint(v.v[4]);
    w.w = ((unsigned long long)__float_as_uint(v.v[7]) << 32) | __float_as_uint(v.v[6]);
    if (p) *reinterpret_cast<ulonglong4_32a*>(a) = w;
}
DEV void st8_if(bool p, double* a, const V8<double>& v) {
    if (p) {
        reinterpret_cast<double4_32a*>(a)[0] = double4_32a{v.v[0], v.v[1], v.v[2], v.v[3]};
        reinterpret_cast<double4_32a*>(a)[1] = double4_32a{v.v[4], v.v[5], v.v[6], v.v[7]};
    }
}
template <class T> DEV void rec_store(bool p, T* rec, size_t cell, int slot, const Al<T>& x) {
    V8<T> q;
#pragma unroll
    for (int a = 0; a < 8; a++) q.v[a] = x.a[a];
    st8_if(p, rec_at(rec, cell, slot), q);
}
// rows 0, 1 of a link into two groups (entries 0..3, then 4, 5, and two unused reals)
template <class T> DEV void rec_store_link(bool p, T* rec, size_t cell, int slot, const M3<T>& U) {
    V8<T> a, b;
#pragma unroll
    for (int e = 0; e < 4; e++) {
        a.v[2 * e] = U.m[e / 3][e % 3].r;
        a.v[2 * e + 1] = U.m[e / 3][e % 3].i;
    }
    b.v[0] = U.m[1][1].r; b.v[1] = U.m[1][1].i; b.v[2] = U.m[1][2].r; b.v[3] = U.m[1][2].i;
    b.v[4] = b.v[5] = b.v[6] = b.v[7] = T(0);
    st8_if(p, rec_at(rec, cell, slot), a);
    st8_if(p, rec_at(rec, cell, slot + 1), b);
}

// One tile [x0, x0+TX) x [y0, y0+TY) of one step: kick at tau_n, drift with tau_{n+1/2}.
// REC: also the gather records of the occupied cells (StepArgs::rec); PLAQ: also the
// plaquettes into the source buffer's last group (StepArgs::plaq, the one-event step,
// whose push reads them); the field arithmetic is the same with and without either.
template <class T, int TX, int TY, bool CG = false, bool REC = false, bool PLAQ = false>
DEV void field_tile(const StepArgs<T>& A, int x0, int y0, unsigned char* smem_raw) {
    using G = RecTile<T, TX, TY>;
    constexpr int HX = G::HX, HS = G::HS, FX = G::FX, FS = G::FS;
    T* sUx = reinterpret_cast<T*>(smem_raw);  // [HS][REC_L]  U_x
    T* sUy = sUx + REC_L * HS;                // [HS][REC_L]  U_y
    T* sP = sUy + REC_L * HS;                 // [HS][REC_A]  phi
    T* sF = sP + REC_A * HS;                  // [FS][REC_A]  ImTL of the plaquette
    const int n = A.n;
    const size_t ns = (size_t)n * n;
    const int tid = threadIdx.y * TX + threadIdx.x;
    const T* __restrict__ src = A.src;

    // own E, pi: issue the loads early
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    const bool active = (x < n) && (y < n);
    const size_t s = active ? (size_t)x + (size_t)n * y : 0;
    Al<T> Ex = load_alg<T, CG>(src, ns, P_EX, s), Ey = load_alg<T, CG>(src, ns, P_EY, s), pi = load_alg<T, CG>(src, ns, P_PI, s);

    // phase 1: links (completed to 3 rows) and phi of the tile plus a one-site halo.
    // Every load of the thread is issued before the first store, so the CTA waits for
    // memory once per tile, not once per pass over the halo.
    {
        constexpr int NT = TX * TY, NIT = (HS + NT - 1) / NT;
        V8<T> raw[NIT][4];
#pragma unroll
        for (int it = 0; it < NIT; it++) {
            const int h = tid + it * NT;
            if (h < HS) {
                const int hx = h % HX, hy = h / HX;
                const size_t g = (size_t)wrapi(x0 - 1 + hx, n) + (size_t)n * wrapi(y0 - 1 + hy, n);
#pragma unroll
                for (int k = 0; k < 3; k++) raw[it][k] = ld8<CG>(src + fidx(8 * k, g, ns));
                raw[it][3] = ld8<CG>(src + fidx(P_PHI, g, ns));
            }
        }
#pragma unroll
        for (int it = 0; it < NIT; it++) {
            const int h = tid + it * NT;
            if (h < HS) {
                M3<T> ux, uy;
                links_from_groups(raw[it][0], raw[it][1], raw[it][2], ux, uy);
                rec_put_link(sUx, h, ux);
                rec_put_link(sUy, h, uy);
                Al<T> ph;
#pragma unroll
                for (int a = 0; a < 8; a++) ph.a[a] = raw[it][3].v[a];
                rec_put_alg(sP, h, ph);
            }
        }
    }
    __syncthreads();

    // phase 2: ImTL P(x) for x in [x0-1, x0+TX) x [y0-1, y0+TY).  The plaquettes beyond
    // the first TX*TY go to the threads that loaded one halo site fewer in phase 1, so that
    // no thread does a second round of both before the barrier.
    constexpr int NT2 = TX * TY, R1 = HS > NT2 ? (HS - NT2) % NT2 : 0;
    for (int i = (tid + NT2 - R1) % NT2; i < FS; i += NT2) {
        const int fx = i % FX, fy = i / FX;
        const int h = fy * HX + fx;
        const M3<T> a1 = mul(rec_link(sUx, h), rec_link(sUy, h + 1));
        const M3<T> b1 = mul(rec_link(sUy, h), rec_link(sUx, h + HX));
        rec_put_alg(sF, i, im_tl(mul_nd(a1, b1)));
    }
    __syncthreads();
    if (!active) return;

    // phase 3: kick and drift of the own site
    const int h = (threadIdx.y + 1) * HX + threadIdx.x + 1;
    const int f = (threadIdx.y + 1) * FX + threadIdx.x + 1;
    const Al<T> phi = rec_alg(sP, h);
    const T dt = A.dtau, tb = A.tb, tp = A.tp;
    // REC: the occupancy stamps of the own cell and of the cells +x, +y (whose records
    // take this site's neighbour pieces), loaded here and first used after the first
    // transport, so that their latency is hidden and no register holds them through
    // phases 1-2.  rm: bit 0 this thread writes its own cell's record, bit 1 the pieces
    // of cell +x, bit 2 those of cell +y; bits 3 and 4 mark a site on the last column or
    // row (the +x, +y neighbours wrap), so that no coordinate stays live for the stores.
    unsigned rm = (x == n - 1 ? 8u : 0u) | (y == n - 1 ? 16u : 0u);
#define GL_CELL_XP ((rm & 8u) ? s - (size_t)(n - 1) : s + 1)
#define GL_CELL_YP ((rm & 16u) ? s - (size_t)n * (n - 1) : s + (size_t)n)
    int o0 = 0, ox = 0, oy = 0;
    if constexpr (REC) {
        const int* occ = A.occ;
        o0 = __ldg(occ + s);
        ox = __ldg(occ + GL_CELL_XP);
        oy = __ldg(occ + GL_CELL_YP);
    }
    // Each link is read from shared memory where it is used and its terms are folded
    // into the increments at once, which keeps few values live per thread.
    Al<T> dEx, dEy, dpi;
    {  // forward x link: U phi(x+x) U^dag, and its commutator with phi (E_x)
        const Al<T> psx = conj_alg(rec_link(sUx, h), rec_alg(sP, h + 1));
        if constexpr (REC) {
            const int ep = A.epoch;
            rm |= A.all_rec ? 7u : ((o0 == ep ? 1u : 0u) | (ox == ep ? 2u : 0u) | (oy == ep ? 4u : 0u));
            rec_store((rm & 1u) != 0, A.rec, s, R_PHI, phi);
            rec_store((rm & 1u) != 0, A.rec, s, R_PSX, psx);
        }
        const Al<T> cm = icomm(phi, psx);
#pragma unroll
        for (int a = 0; a < 8; a++) { dpi.a[a] = psx.a[a]; dEx.a[a] = -tp * cm.a[a]; }
    }
    {  // forward y link (E_y)
        const Al<T> psy = conj_alg(rec_link(sUy, h), rec_alg(sP, h + HX));
        if constexpr (REC) rec_store((rm & 1u) != 0, A.rec, s, R_PSY, psy);
        const Al<T> cm = icomm(phi, psy);
#pragma unroll
        for (int a = 0; a < 8; a++) { dpi.a[a] += psy.a[a]; dEy.a[a] = -tp * cm.a[a]; }
    }
    {  // backward x link: phi(x-x) and the plaquette at x-x carried to x
        const M3<T> uxm = rec_link(sUx, h - 1);
        const Al<T> chx = transport_alg(uxm, rec_alg(sP, h - 1));
        const Al<T> t2 = transport_alg(uxm, rec_alg(sF, f - 1));
        if constexpr (REC) {
            rec_store((rm & 1u) != 0, A.rec, s, R_CHX, chx);
            rec_store((rm & 1u) != 0, A.rec, s, R_T2, t2);
        }
#pragma unroll
        for (int a = 0; a < 8; a++) { dpi.a[a] += chx.a[a]; dEy.a[a] -= tb * t2.a[a]; }
    }
    {  // backward y link: phi(x-y) and the plaquette at x-y carried to x
        const M3<T> uym = rec_link(sUy, h - HX);
        const Al<T> chy = transport_alg(uym, rec_alg(sP, h - HX));
        const Al<T> t1 = transport_alg(uym, rec_alg(sF, f - FX));
        if constexpr (REC) {
            rec_store((rm & 1u) != 0, A.rec, s, R_CHY, chy);
            rec_store((rm & 1u) != 0, A.rec, s, R_T1, t1);
            rec_store((rm & 2u) != 0, A.rec, GL_CELL_XP, R_T1L, t1);
        }
#pragma unroll
        for (int a = 0; a < 8; a++) { dpi.a[a] += chy.a[a]; dEx.a[a] += tb * t1.a[a]; }
    }
    {
        const Al<T> F0 = rec_alg(sF, f);
        if constexpr (PLAQ) store_alg(A.plaq, ns, P_F, s, F0);  // for the push of this step
        if constexpr (REC) {
            // the same updates, one field at a time, each followed by its time average
            // (E_{n-1/2} + E_{n+1/2}) / 2 formed exactly as the unfused gather forms it
            rec_store((rm & 1u) != 0, A.rec, s, R_F0, F0);
            {
                Al<T> z;
#pragma unroll
                for (int a = 0; a < 8; a++) z.a[a] = T(0);
                rec_store((rm & 1u) != 0, A.rec, s, R_PAD0, z);
            }
            Al<T> av;
#pragma unroll
            for (int a = 0; a < 8; a++) {
                const T o = Ex.a[a];
                Ex.a[a] += dt * (dEx.a[a] - tb * F0.a[a]);
                av.a[a] = T(0.5) * (o + Ex.a[a]);
            }
            rec_store((rm & 1u) != 0, A.rec, s, R_EX, av);
            rec_store((rm & 2u) != 0, A.rec, GL_CELL_XP, R_EXL, av);
#pragma unroll
            for (int a = 0; a < 8; a++) {
                const T o = Ey.a[a];
                Ey.a[a] += dt * (dEy.a[a] + tb * F0.a[a]);
                av.a[a] = T(0.5) * (o + Ey.a[a]);
            }
            rec_store((rm & 1u) != 0, A.rec, s, R_EY, av);
            rec_store((rm & 4u) != 0, A.rec, GL_CELL_YP, R_EYB, av);
#pragma unroll
            for (int a = 0; a < 8; a++) {
                const T o = pi.a[a];
                pi.a[a] += dt * tp * (dpi.a[a] - T(4) * phi.a[a]);
                av.a[a] = T(0.5) * (o + pi.a[a]);
            }
            rec_store((rm & 1u) != 0, A.rec, s, R_PI, av);
        } else {
#pragma unroll
            for (int a = 0; a < 8; a++) {
                Ex.a[a] += dt * (dEx.a[a] - tb * F0.a[a]);
                Ey.a[a] += dt * (dEy.a[a] + tb * F0.a[a]);
                pi.a[a] += dt * tp * (dpi.a[a] - T(4) * phi.a[a]);
            }
        }
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
    M3<T> Vn[2];
#pragma unroll
    for (int d = 0; d < 2; d++) {
        Al<T> e = d == 0 ? Ex : Ey;
#pragma unroll
        for (int a = 0; a < 8; a++) e.a[a] *= A.ue;
        const M3<T> W = expi(herm(e));
        const M3<T> U = rec_link(d == 0 ? sUx : sUy, h);
        if constexpr (REC) {  // U_n of this site for the record of cell +x (U_x) or +y (U_y)
            if (d == 0) rec_store_link((rm & 2u) != 0, A.rec, GL_CELL_XP, R_UXL, U);
            else {
                rec_store_link((rm & 4u) != 0, A.rec, GL_CELL_YP, R_UYB, U);
                Al<T> z;
#pragma unroll
                for (int a = 0; a < 8; a++) z.a[a] = T(0);
                rec_store((rm & 4u) != 0, A.rec, GL_CELL_YP, R_PAD1, z);
            }
        }
        M3<T> V;
#pragma unroll
        for (int r = 0; r < 2; r++)
#pragma unroll
            for (int c = 0; c < 3; c++)
                V.m[r][c] = val(cmac(cmac(cmul(W.m[r][0], U.m[0][c]), W.m[r][1], U.m[1][c]), W.m[r][2], U.m[2][c]));
        if (A.reunit == 1) reunit_rows(V);
        else if (A.reunit == 2 && sizeof(T) == 4) renorm_rows(V);
        Vn[d] = V;
    }
    store_links(dst, ns, s, Vn[0], Vn[1]);
#undef GL_CELL_XP
#undef GL_CELL_YP
}

}  // namespace glasma
