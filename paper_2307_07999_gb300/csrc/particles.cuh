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
        for (int j = 0; j < 3; j++) {
            cx<T> s = mk(T(0), T(0));
            fmca_(s, A.m[0][i], B.m[0][j]);
            fmca_(s, A.m[1][i], B.m[1][j]);
            fmca_(s, A.m[2][i], B.m[2][j]);
            C.m[i][j] = s;
        }
    return C;
}
template <class T> DEV T dot8(const Al<T>& a, const Al<T>& b) {
    T s = T(0);
#pragma unroll
    for (int k = 0; k < 8; k++) s = fma(a.a[k], b.a[k], s);
    return s;
}

// site-centred fields at cell (cx, cy) for the push of step n:
// F[0..2] = E_x, E_y, E_z ; F[3..5] = B_x, B_y, B_z   (contracted with Q on return)
template <class T>
DEV void gather_qf(const PushArgs<T>& A, int cx, int cy, const Al<T>& q, T qE[3], T qB[3]) {
    const int n = A.n;
    const size_t ns = (size_t)n * n;
    const int xm = cx == 0 ? n - 1 : cx - 1, xp = cx == n - 1 ? 0 : cx + 1;
    const int ym = cy == 0 ? n - 1 : cy - 1, yp = cy == n - 1 ? 0 : cy + 1;
    const size_t c = cx + (size_t)n * cy;
    const size_t cxm = xm + (size_t)n * cy, cxp = xp + (size_t)n * cy;
    const size_t cym = cx + (size_t)n * ym, cyp = cx + (size_t)n * yp;
    const T* fo = A.fo;
    const T* fn = A.fn;
    const T half = T(0.5);
    const M3<T> ux_c = load_link(fo, ns, P_UX, c), uy_c = load_link(fo, ns, P_UY, c);
    const M3<T> ux_xm = load_link(fo, ns, P_UX, cxm), uy_ym = load_link(fo, ns, P_UY, cym);
    // electric: the two links touching c, time-centred, transported to c
    {
        Al<T> ec, em;
#pragma unroll
        for (int a = 0; a < 8; a++) {
            ec.a[a] = half * (__ldg(fo + (size_t)(P_EX + a) * ns + c) + __ldg(fn + (size_t)(P_EX + a) * ns + c));
            em.a[a] = half * (__ldg(fo + (size_t)(P_EX + a) * ns + cxm) + __ldg(fn + (size_t)(P_EX + a) * ns + cxm));
        }
        const Al<T> t = transport_alg(ux_xm, em);
        qE[0] = half * (dot8(q, ec) + dot8(q, t)) / A.te;
    }
    {
        Al<T> ec, em;
#pragma unroll
        for (int a = 0; a < 8; a++) {
            ec.a[a] = half * (__ldg(fo + (size_t)(P_EY + a) * ns + c) + __ldg(fn + (size_t)(P_EY + a) * ns + c));
            em.a[a] = half * (__ldg(fo + (size_t)(P_EY + a) * ns + cym) + __ldg(fn + (size_t)(P_EY + a) * ns + cym));
        }
        const Al<T> t = transport_alg(uy_ym, em);
        qE[1] = half * (dot8(q, ec) + dot8(q, t)) / A.te;
    }
    {
        T s = T(0);
#pragma unroll
        for (int a = 0; a < 8; a++)
            s = fma(q.a[a], half * (__ldg(fo + (size_t)(P_PI + a) * ns + c) + __ldg(fn + (size_t)(P_PI + a) * ns + c)), s);
        qE[2] = s;
    }
    // magnetic from phi: covariant central differences
    {
        const Al<T> fw = conj_alg(ux_c, load_alg(fo, ns, P_PHI, cxp));
        const Al<T> bw = transport_alg(ux_xm, load_alg(fo, ns, P_PHI, cxm));
        qB[1] = half * (dot8(q, fw) - dot8(q, bw)) / A.te;    // B_y = +D_x phi / tau
    }
    {
        const Al<T> fw = conj_alg(uy_c, load_alg(fo, ns, P_PHI, cyp));
        const Al<T> bw = transport_alg(uy_ym, load_alg(fo, ns, P_PHI, cym));
        qB[0] = -half * (dot8(q, fw) - dot8(q, bw)) / A.te;   // B_x = -D_y phi / tau
    }
    // B_z = -F_xy, F_xy = clover average of the four plaquettes based at c
    {
        const size_t cxpym = xp + (size_t)n * ym, cxmyp = xm + (size_t)n * yp, cxmym = xm + (size_t)n * ym;
        Al<T> acc;
        {   // +x,+y
            const M3<T> P = mul_nd(mul(ux_c, load_link(fo, ns, P_UY, cxp)), mul(uy_c, load_link(fo, ns, P_UX, cyp)));
            acc = im_tl(P);
        }
        {   // +y,-x: U_y(c) [U_y(c-x) U_x(c-x+y)]^dag U_x(c-x)
            const M3<T> B = mul(load_link(fo, ns, P_UY, cxm), load_link(fo, ns, P_UX, cxmyp));
            const Al<T> t = im_tl(mul(mul_nd(uy_c, B), ux_xm));
#pragma unroll
            for (int a = 0; a < 8; a++) acc.a[a] += t.a[a];
        }
        {   // -x,-y: [U_y(c-x-y) U_x(c-x)]^dag [U_x(c-x-y) U_y(c-y)]
            const M3<T> B1 = mul(load_link(fo, ns, P_UY, cxmym), ux_xm);
            const M3<T> B2 = mul(load_link(fo, ns, P_UX, cxmym), uy_ym);
            const Al<T> t = im_tl(mul_dn(B1, B2));
#pragma unroll
            for (int a = 0; a < 8; a++) acc.a[a] += t.a[a];
        }
        {   // -y,+x: U_y(c-y)^dag [U_x(c-y) U_y(c+x-y)] U_x(c)^dag
            const M3<T> B = mul(load_link(fo, ns, P_UX, cym), load_link(fo, ns, P_UY, cxpym));
            const Al<T> t = im_tl(mul_nd(mul_dn(uy_ym, B), ux_c));
#pragma unroll
            for (int a = 0; a < 8; a++) acc.a[a] += t.a[a];
        }
        qB[2] = -T(0.25) * dot8(q, acc);
    }
}

template <class T> DEV T clamp_below_one(T v);
template <> DEV float clamp_below_one<float>(float v) { return fminf(v, 0.99999994f); }
template <> DEV double clamp_below_one<double>(double v) { return fmin(v, 0.99999999999999989); }

// one particle: gather, kick, drift, color transport; returns its broadening terms
template <class T>
DEV void push_one(const PushArgs<T>& A, int j, double& sx, double& sy, double& sz, double& sc) {
    const PartSoA<T>& P = A.P;
    const int n = A.n;
    const size_t ns = (size_t)n * n;
    const int cell = P.cell[j];
    int cx = cell % n, cy = cell / n;
    Al<T> q;
#pragma unroll
    for (int a = 0; a < 8; a++) q.a[a] = P.Q[(size_t)a * P.qs + j];
    T qE[3], qB[3];
    gather_qf(A, cx, cy, q, qE, qB);
    const T p0x = P.p0x[j], p0y = P.p0y[j];
    T dpx = P.dpx[j], dpy = P.dpy[j], pz = P.peta[j];
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
    T ox = P.ox[j] + A.dtau * px * iptn;
    T oy = P.oy[j] + A.dtau * py * iptn;
    const T deta = A.dtau * pz * iptn / A.teh;
    // color: rotation along eta at the old cell, then across the x face, then the y face
    {
        Al<T> e;
        const Al<T> ph = load_alg(A.fo, ns, P_PHI, (size_t)cell);
#pragma unroll
        for (int a = 0; a < 8; a++) e.a[a] = -deta * ph.a[a];
        q = alg(conj_by(expi(herm(e)), herm(q)));
    }
    int nx = cx, ny = cy;
    if (ox >= T(1)) {
        q = transport_alg(load_link(A.fo, ns, P_UX, (size_t)cell), q);
        ox -= T(1);
        nx = cx == n - 1 ? 0 : cx + 1;
    } else if (ox < T(0)) {
        nx = cx == 0 ? n - 1 : cx - 1;
        q = conj_alg(load_link(A.fo, ns, P_UX, nx + (size_t)n * cy), q);
        ox = clamp_below_one(ox + T(1));
    }
    if (oy >= T(1)) {
        q = transport_alg(load_link(A.fo, ns, P_UY, nx + (size_t)n * cy), q);
        oy -= T(1);
        ny = cy == n - 1 ? 0 : cy + 1;
    } else if (oy < T(0)) {
        ny = cy == 0 ? n - 1 : cy - 1;
        q = conj_alg(load_link(A.fo, ns, P_UY, nx + (size_t)n * ny), q);
        oy = clamp_below_one(oy + T(1));
    }
    const T eta = P.eta[j] + deta;
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

// warp -> block -> one FP64 atomic per block and term (blockDim.x <= 256)
DEV void block_acc4(double sx, double sy, double sz, double sc, double* acc) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_down_sync(0xffffffffu, sx, o);
        sy += __shfl_down_sync(0xffffffffu, sy, o);
        sz += __shfl_down_sync(0xffffffffu, sz, o);
        sc += __shfl_down_sync(0xffffffffu, sc, o);
    }
    __shared__ double red[4][8];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { red[0][w] = sx; red[1][w] = sy; red[2][w] = sz; red[3][w] = sc; }
    __syncthreads();
    if (threadIdx.x < 4) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += red[threadIdx.x][k];
        atomicAdd(acc + threadIdx.x, t);
    }
}

template <class T>
__global__ void __launch_bounds__(256) k_push(PushArgs<T> A) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    double sx = 0.0, sy = 0.0, sz = 0.0, sc = 0.0;
    if (j < A.np) push_one(A, j, sx, sy, sz, sc);
    block_acc4(sx, sy, sz, sc, A.acc);
}

// batched over events: one 256-particle block per item; args[ev] of this step
// (acc == nullptr marks an event whose particles are not pushed at this step)
struct PushItem { int ev, j0; };
template <class T>
__global__ void __launch_bounds__(256) k_push_batched(const PushArgs<T>* __restrict__ args,
                                                      const PushItem* __restrict__ items) {
    const PushItem it = items[blockIdx.x];
    const PushArgs<T> A = args[it.ev];
    if (A.acc == nullptr) return;
    const int j = it.j0 + threadIdx.x;
    double sx = 0.0, sy = 0.0, sz = 0.0, sc = 0.0;
    if (j < A.np) push_one(A, j, sx, sy, sz, sc);
    block_acc4(sx, sy, sz, sc, A.acc);
}

// ---------------------------------------------------------------- counting sort by cell
__global__ void k_cell_count(const int* __restrict__ cell, int np, int* __restrict__ count) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < np) atomicAdd(count + cell[j], 1);
}
// exclusive scan, three passes: per-block scan with block totals, scan of the totals, add
__global__ void k_scan_block(const int* __restrict__ in, int* __restrict__ out, int* __restrict__ totals, int len) {
    __shared__ int buf[1024];
    const int i = blockIdx.x * 1024 + threadIdx.x;
    const int v = i < len ? in[i] : 0;
    buf[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int t = threadIdx.x >= o ? buf[threadIdx.x - o] : 0;
        __syncthreads();
        buf[threadIdx.x] += t;
        __syncthreads();
    }
    if (i < len) out[i] = buf[threadIdx.x] - v;
    if (threadIdx.x == 1023) totals[blockIdx.x] = buf[1023];
}
__global__ void k_scan_totals(int* totals, int nb) {
    // one thread: nb is at most a few thousand
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int run = 0;
        for (int b = 0; b < nb; b++) { const int t = totals[b]; totals[b] = run; run += t; }
    }
}
__global__ void k_scan_add(int* __restrict__ out, const int* __restrict__ totals, int len) {
    const int i = blockIdx.x * 1024 + threadIdx.x;
    if (i < len) out[i] += totals[blockIdx.x];
}
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
