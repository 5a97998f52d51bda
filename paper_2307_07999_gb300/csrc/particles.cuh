// Colored particle-in-cell push of test particles under Wong's equations
// (Sec. 1 "Probes in Glasma", Eq. 2 of arXiv:2307.07999) and the momentum-
// broadening sums of Sec. 2 ("Quantifying the effect of Glasma").
//
// Particle state (structure of arrays, n_p entries each):
//   cell (int32, x + n*y), pid (int32, original index), ox, oy (offsets in the
//   cell, [0,1)), eta, p0x, p0y, p0z (lab momentum at formation), dpx, dpy
//   (px = p0x + dpx, py = p0y + dpy), peta (tau * p^eta), Q^a (8 planes).
// Keeping the transverse momentum as p0 + dp and the position as cell + offset
// keeps FP32 round-off relative to the change, not to the absolute value.
#pragma once
#include "field.cuh"

namespace glasma {

template <class T> struct PartSoA {
    int* cell; int* pid;
    T *ox, *oy, *eta, *p0x, *p0y, *p0z, *dpx, *dpy, *peta, *Q;  // Q: 8 planes, stride qs
    size_t qs;
};

template <class T> struct PushArgs {
    const T* fo;   // fields at step n   (U_n, phi_n, E_{n-1/2}, pi_{n-1/2})
    const T* fn;   // fields at step n+1 (E_{n+1/2}, pi_{n+1/2} used)
    int n;
    PartSoA<T> P;
    int np;
    T dtau;
    T te;          // tau_n (expanding) or 1: divides E_i and D_i phi
    T ichr;        // 1/tau_n (expanding, Christoffel term) or 0
    T teh;         // tau_{n+1/2} (expanding) or 1: eta drift
    T mass;
    int expanding;
    double* acc;   // this step's row: {sum dpx^2, sum dpy^2, sum dpz^2, count}
};

template <class T> DEV M3<T> mul_dn(const M3<T>& A, const M3<T>& B) {  // A^dag B
    M3<T> C;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++)
            C.m[i][j] = val(ccmac(ccmac(ccmul(A.m[0][i], B.m[0][j]), A.m[1][i], B.m[1][j]), A.m[2][i], B.m[2][j]));
    return C;
}
template <class T> DEV T dot8(const Al<T>& a, const Al<T>& b) {
    T s = T(0);
#pragma unroll
    for (int k = 0; k < 8; k++) s = fma(a.a[k], b.a[k], s);
    return s;
}

template <class T> DEV T clamp_below_one(T v);
template <> DEV float clamp_below_one<float>(float v) { return fminf(v, 0.99999994f); }
template <> DEV double clamp_below_one<double>(double v) { return fmin(v, 0.99999999999999989); }

// Field source of the unfused push: links, phi and time-averaged E, pi read from
// the two global field buffers of step n.  Cells are given as (x, y) with the
// neighbours already wrapped periodically.
template <class T, bool CG = false> struct GlobalSrc {
    const T* fo;
    const T* fn;
    int n;
    size_t ns;
    DEV size_t at(int x, int y) const { return (size_t)x + (size_t)n * y; }
    DEV M3<T> link(int d, int x, int y) const { return load_link<T, CG>(fo, ns, d == 0 ? P_UX : P_UY, at(x, y)); }
    DEV void links(int x, int y, M3<T>& ux, M3<T>& uy) const { load_links<T, CG>(fo, ns, at(x, y), ux, uy); }
    DEV Al<T> phi(int x, int y) const { return load_alg<T, CG>(fo, ns, P_PHI, at(x, y)); }
    // (E_i(tau_{n-1/2}) + E_i(tau_{n+1/2})) / 2 on the link (x, y) -> (x, y) + i
    DEV Al<T> eavg(int d, int x, int y) const { return avg(d == 0 ? P_EX : P_EY, at(x, y)); }
    DEV Al<T> piavg(int x, int y) const { return avg(P_PI, at(x, y)); }
    DEV Al<T> avg(int p, size_t s) const {
        Al<T> e = load_alg<T, CG>(fo, ns, p, s);
        const Al<T> b = load_alg<T, CG>(fn, ns, p, s);
#pragma unroll
        for (int a = 0; a < 8; a++) e.a[a] = T(0.5) * (e.a[a] + b.a[a]);
        return e;
    }
};

// Q-contracted site-centred fields at cell (cx, cy) for the push of step n:
// qE = Q.(E_x, E_y, E_z), qB = Q.(B_x, B_y, B_z)
template <class T, class S>
DEV void gather_qf_src(const S& F, int n, T te, int cx, int cy, const Al<T>& q, T qE[3], T qB[3]) {
    const int xm = cx == 0 ? n - 1 : cx - 1, xp = cx == n - 1 ? 0 : cx + 1;
    const int ym = cy == 0 ? n - 1 : cy - 1, yp = cy == n - 1 ? 0 : cy + 1;
    const T half = T(0.5);
    // cells whose two links are both used load them together (three sectors in FP32)
    M3<T> ux_c, uy_c, ux_xm, uy_xm, ux_ym, uy_ym;
    F.links(cx, cy, ux_c, uy_c);
    F.links(xm, cy, ux_xm, uy_xm);
    F.links(cx, ym, ux_ym, uy_ym);
    // electric: the two links touching c, time-centred, transported to c
    {
        const Al<T> t = transport_alg(ux_xm, F.eavg(0, xm, cy));
        qE[0] = half * (dot8(q, F.eavg(0, cx, cy)) + dot8(q, t)) / te;
    }
    {
        const Al<T> t = transport_alg(uy_ym, F.eavg(1, cx, ym));
        qE[1] = half * (dot8(q, F.eavg(1, cx, cy)) + dot8(q, t)) / te;
    }
    qE[2] = dot8(q, F.piavg(cx, cy));
    // magnetic from phi: covariant central differences
    {
        const Al<T> fw = conj_alg(ux_c, F.phi(xp, cy));
        const Al<T> bw = transport_alg(ux_xm, F.phi(xm, cy));
        qB[1] = half * (dot8(q, fw) - dot8(q, bw)) / te;    // B_y = +D_x phi / tau
    }
    {
        const Al<T> fw = conj_alg(uy_c, F.phi(cx, yp));
        const Al<T> bw = transport_alg(uy_ym, F.phi(cx, ym));
        qB[0] = -half * (dot8(q, fw) - dot8(q, bw)) / te;   // B_x = -D_y phi / tau
    }
    // B_z = -F_xy, F_xy = clover average of the four plaquettes based at c
    {
        Al<T> acc = im_tl(mul_nd(mul(ux_c, F.link(1, xp, cy)), mul(uy_c, F.link(0, cx, yp))));  // +x,+y
        {   // +y,-x: U_y(c) [U_y(c-x) U_x(c-x+y)]^dag U_x(c-x)
            const M3<T> B = mul(uy_xm, F.link(0, xm, yp));
            const Al<T> t = im_tl(mul(mul_nd(uy_c, B), ux_xm));
#pragma unroll
            for (int a = 0; a < 8; a++) acc.a[a] += t.a[a];
        }
        {   // -x,-y: [U_y(c-x-y) U_x(c-x)]^dag [U_x(c-x-y) U_y(c-y)]
            M3<T> ux_xmym, uy_xmym;
            F.links(xm, ym, ux_xmym, uy_xmym);
            const M3<T> B1 = mul(uy_xmym, ux_xm);
            const M3<T> B2 = mul(ux_xmym, uy_ym);
            const Al<T> t = im_tl(mul_dn(B1, B2));
#pragma unroll
            for (int a = 0; a < 8; a++) acc.a[a] += t.a[a];
        }
        {   // -y,+x: U_y(c-y)^dag [U_x(c-y) U_y(c+x-y)] U_x(c)^dag
            const M3<T> B = mul(ux_ym, F.link(1, xp, ym));
            const Al<T> t = im_tl(mul_nd(mul_dn(uy_ym, B), ux_c));
#pragma unroll
            for (int a = 0; a < 8; a++) acc.a[a] += t.a[a];
        }
        qB[2] = -T(0.25) * dot8(q, acc);
    }
}

template <class T>
DEV void gather_qf(const PushArgs<T>& A, int cx, int cy, const Al<T>& q, T qE[3], T qB[3]) {
    GlobalSrc<T> F{A.fo, A.fn, A.n, (size_t)A.n * A.n};
    gather_qf_src(F, A.n, A.te, cx, cy, q, qE, qB);
}


// one particle: gather, kick, drift, color transport; returns its broadening terms
template <class T, class S, bool CG = false>
DEV void push_one_src(const PushArgs<T>& A, const S& F, int j, double& sx, double& sy, double& sz, double& sc) {
    const PartSoA<T>& P = A.P;
    const int n = A.n;
    const int cell = CG ? __ldcg(P.cell + j) : P.cell[j];
    int cx = cell % n, cy = cell / n;
    Al<T> q;
#pragma unroll
    for (int a = 0; a < 8; a++) q.a[a] = CG ? __ldcg(P.Q + (size_t)a * P.qs + j) : P.Q[(size_t)a * P.qs + j];
    T qE[3], qB[3];
    gather_qf_src(F, n, A.te, cx, cy, q, qE, qB);
    const T p0x = P.p0x[j], p0y = P.p0y[j];  // constant during a run
    T dpx = CG ? __ldcg(P.dpx + j) : P.dpx[j], dpy = CG ? __ldcg(P.dpy + j) : P.dpy[j];
    T pz = CG ? __ldcg(P.peta + j) : P.peta[j];
    const T m2 = A.mass * A.mass;
    T px = p0x + dpx, py = p0y + dpy;
    const T pt = sqrt(m2 + px * px + py * py + pz * pz);
    const T ipt = pt > T(0) ? T(1) / pt : T(0);
    const T fx = qE[0] + (py * qB[2] - pz * qB[1]) * ipt;
    const T fy = qE[1] + (pz * qB[0] - px * qB[2]) * ipt;
    const T fz = qE[2] + (px * qB[1] - py * qB[0]) * ipt - pz * A.ichr;
    dpx += A.dtau * fx;
    dpy += A.dtau * fy;
    pz += A.dtau * fz;
    px = p0x + dpx;
    py = p0y + dpy;
    const T ptn = sqrt(m2 + px * px + py * py + pz * pz);
    const T iptn = ptn > T(0) ? T(1) / ptn : T(0);
    T ox = (CG ? __ldcg(P.ox + j) : P.ox[j]) + A.dtau * px * iptn;
    T oy = (CG ? __ldcg(P.oy + j) : P.oy[j]) + A.dtau * py * iptn;
    const T deta = A.dtau * pz * iptn / A.teh;
    // color: rotation along eta at the old cell, then across the x face, then the y face
    {
        Al<T> e;
        const Al<T> ph = F.phi(cx, cy);
#pragma unroll
        for (int a = 0; a < 8; a++) e.a[a] = -deta * ph.a[a];
        q = alg(conj_by(expi(herm(e)), herm(q)));
    }
    int nx = cx, ny = cy;
    if (ox >= T(1)) {
        q = transport_alg(F.link(0, cx, cy), q);
        ox -= T(1);
        nx = cx == n - 1 ? 0 : cx + 1;
    } else if (ox < T(0)) {
        nx = cx == 0 ? n - 1 : cx - 1;
        q = conj_alg(F.link(0, nx, cy), q);
        ox = clamp_below_one(ox + T(1));
    }
    if (oy >= T(1)) {
        q = transport_alg(F.link(1, nx, cy), q);
        oy -= T(1);
        ny = cy == n - 1 ? 0 : cy + 1;
    } else if (oy < T(0)) {
        ny = cy == 0 ? n - 1 : cy - 1;
        q = conj_alg(F.link(1, nx, ny), q);
        oy = clamp_below_one(oy + T(1));
    }
    const T eta = (CG ? __ldcg(P.eta + j) : P.eta[j]) + deta;
    P.cell[j] = nx + n * ny;
    P.ox[j] = ox;
    P.oy[j] = oy;
    P.eta[j] = eta;
    P.dpx[j] = dpx;
    P.dpy[j] = dpy;
    P.peta[j] = pz;
#pragma unroll
    for (int a = 0; a < 8; a++) P.Q[(size_t)a * P.qs + j] = q.a[a];
    // broadening terms: dp_i^2 = p_i^2 - p_i(tau_form)^2, lab p_z
    const double pzl = A.expanding ? (double)ptn * sinh((double)eta) + (double)pz * cosh((double)eta)
                                   : (double)pz;
    const double p0z = (double)P.p0z[j];
    sx = (double)dpx * (2.0 * (double)p0x + (double)dpx);
    sy = (double)dpy * (2.0 * (double)p0y + (double)dpy);
    sz = pzl * pzl - p0z * p0z;
    sc = 1.0;
}

template <class T, bool CG = false>
DEV void push_one(const PushArgs<T>& A, int j, double& sx, double& sy, double& sz, double& sc) {
    GlobalSrc<T, CG> F{A.fo, A.fn, A.n, (size_t)A.n * A.n};
    push_one_src<T, GlobalSrc<T, CG>, CG>(A, F, j, sx, sy, sz, sc);
}

// warp -> block -> one FP64 atomic per block and term (any block shape, at most 256
// threads, a multiple of 32)
DEV void block_acc4(double sx, double sy, double sz, double sc, double* acc) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_down_sync(0xffffffffu, sx, o);
        sy += __shfl_down_sync(0xffffffffu, sy, o);
        sz += __shfl_down_sync(0xffffffffu, sz, o);
        sc += __shfl_down_sync(0xffffffffu, sc, o);
    }
    __shared__ double red[4][8];
    const int lt = threadIdx.y * blockDim.x + threadIdx.x;
    const int nw = (blockDim.x * blockDim.y) >> 5;
    const int w = lt >> 5, l = lt & 31;
    if (l == 0) { red[0][w] = sx; red[1][w] = sy; red[2][w] = sz; red[3][w] = sc; }
    __syncthreads();
    if (lt < 4) {
        double t = 0.0;
        for (int k = 0; k < nw; k++) t += red[lt][k];
        atomicAdd(acc + lt, t);
    }
}

template <class T>
__global__ void __launch_bounds__(256) k_push(PushArgs<T> A) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    double sx = 0.0, sy = 0.0, sz = 0.0, sc = 0.0;
    if (j < A.np) push_one(A, j, sx, sy, sz, sc);
    block_acc4(sx, sy, sz, sc, A.acc);
}

// batched over events: one item per 256 particles of an event, pushed by
// 256 / PUSH_THREADS blocks; args[ev] of this step (acc == nullptr marks an event
// whose particles are not pushed at this step)
#ifndef GLASMA_PUSH_THREADS
#define GLASMA_PUSH_THREADS 256
#endif
#ifndef GLASMA_PUSH_MINB
#define GLASMA_PUSH_MINB 1
#endif
constexpr int PUSH_THREADS = GLASMA_PUSH_THREADS, PUSH_SUB = 256 / GLASMA_PUSH_THREADS;
static_assert(256 % GLASMA_PUSH_THREADS == 0 && GLASMA_PUSH_THREADS % 32 == 0, "push block");
struct PushItem { int ev, j0; };
template <class T>
__global__ void __launch_bounds__(GLASMA_PUSH_THREADS, GLASMA_PUSH_MINB)
k_push_batched(const PushArgs<T>* __restrict__ args, const PushItem* __restrict__ items) {
    const PushItem it = items[blockIdx.x / PUSH_SUB];
    const PushArgs<T> A = args[it.ev];
    if (A.acc == nullptr) return;
    const int j = it.j0 + (int)(blockIdx.x % PUSH_SUB) * PUSH_THREADS + threadIdx.x;
    double sx = 0.0, sy = 0.0, sz = 0.0, sc = 0.0;
    if (j < A.np) push_one(A, j, sx, sy, sz, sc);
    block_acc4(sx, sy, sz, sc, A.acc);
}

// ---------------------------------------------------------------- counting sort by cell
template <class T>
__global__ void k_scatter(PartSoA<T> a, PartSoA<T> b, int np, int* __restrict__ cursor) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= np) return;
    const int c = a.cell[j];
    const int k = atomicAdd(cursor + c, 1);
    b.cell[k] = c; b.pid[k] = a.pid[j];
    b.ox[k] = a.ox[j]; b.oy[k] = a.oy[j]; b.eta[k] = a.eta[j];
    b.p0x[k] = a.p0x[j]; b.p0y[k] = a.p0y[j]; b.p0z[k] = a.p0z[j];
    b.dpx[k] = a.dpx[j]; b.dpy[k] = a.dpy[j]; b.peta[k] = a.peta[j];
#pragma unroll
    for (int q = 0; q < 8; q++) b.Q[(size_t)q * b.qs + k] = a.Q[(size_t)q * a.qs + j];
}

}  // namespace glasma
