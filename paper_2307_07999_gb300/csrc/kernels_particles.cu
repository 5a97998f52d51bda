// Particle kernels: CPIC push with the fused broadening reduction, counting sort
// by cell, Philox initial state (Sec. 1 "Probes in Glasma" and Sec. 2 of
// arXiv:2307.07999), host-layout conversion and the Casimir monitor.
#include <algorithm>
#include <type_traits>

#include "ic.cuh"
#include "internal.h"
#include "particles.cuh"

namespace glasma {

size_t part_bytes(int np, int prec) {
    const size_t rs = prec ? 4 : 8;
    return 2 * align256((size_t)np * 4) + N_PART_REAL_PLANES * align256((size_t)np * rs);
}
PartHost part_layout(void* base, int np, int prec) {
    const size_t rs = prec ? 4 : 8;
    char* p = (char*)base;
    PartHost h;
    h.cell = (int*)p;
    p += align256((size_t)np * 4);
    h.pid = (int*)p;
    p += align256((size_t)np * 4);
    h.planes = p;
    h.pstride = align256((size_t)np * rs) / rs;
    return h;
}
template <class T> static PartSoA<T> soa(const PartHost& h) {
    PartSoA<T> P;
    T* b = (T*)h.planes;
    const size_t ps = h.pstride;
    P.cell = h.cell; P.pid = h.pid;
    P.ox = b; P.oy = b + ps; P.eta = b + 2 * ps; P.p0x = b + 3 * ps; P.p0y = b + 4 * ps; P.p0z = b + 5 * ps;
    P.dpx = b + 6 * ps; P.dpy = b + 7 * ps; P.peta = b + 8 * ps; P.Q = b + 9 * ps;
    P.qs = ps;
    return P;
}
template <class T> static PushArgs<T> push_args(const PushHost& a, const PartHost& h) {
    PushArgs<T> A;
    A.fo = (const T*)a.fo; A.fn = (const T*)a.fn; A.n = a.n;
    A.P = soa<T>(h); A.np = a.np;
    A.dtau = (T)a.dtau; A.te = (T)a.te; A.ichr = (T)a.ichr; A.teh = (T)a.teh; A.mass = (T)a.mass;
    A.expanding = a.expanding; A.acc = a.acc;
    A.boris = a.boris; A.dec0 = (T)a.dec0; A.dec1 = (T)a.dec1;
    A.nsub = a.nsub; A.hsub = (T)a.hsub; A.tau0 = (T)a.tau0; A.interp = a.interp;
    A.rec = (const T*)a.rec; A.occ = a.occ; A.epoch_next = a.epoch_next;
    A.frc = (T*)a.frc;
    return A;
}
size_t record_bytes(int prec) { return (size_t)REC_STRIDE * 8 * (prec ? 4 : 8); }
size_t push_args_size(int prec) { return prec ? sizeof(PushArgs<float>) : sizeof(PushArgs<double>); }
void pack_push_args(int prec, const PushHost& a, const PartHost& P, void* out) {
    if (prec) *(PushArgs<float>*)out = push_args<float>(a, P);
    else *(PushArgs<double>*)out = push_args<double>(a, P);
}
// Batched push kernels, chosen per batch by measurement (glasma_batch_tune):
//   0: 128-thread blocks, 3 per SM, fields read through L1
//   1: 32-thread blocks, 6 per SM, each particle's fields staged in shared memory first
//   2: the fields from the gather records the field launch wrote (PUSH_VARIANT_RECORD)
//   3: split into a force kernel and a move kernel (PUSH_VARIANT_SPLIT)
int push_variants() { return 4; }
#ifndef GLASMA_SPLIT_FORCE_MINB
#define GLASMA_SPLIT_FORCE_MINB 3
#endif
#ifndef GLASMA_SPLIT_MOVE_MINB
#define GLASMA_SPLIT_MOVE_MINB 4
#endif
constexpr int SPLIT_FORCE_MINB = GLASMA_SPLIT_FORCE_MINB, SPLIT_MOVE_MINB = GLASMA_SPLIT_MOVE_MINB;
// shared-memory limit of the staged push (call outside stream capture)
cudaError_t prepare_push_staged() {
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_push_staged<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)push_staged_smem<float>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_push_staged<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)push_staged_smem<double>());
    if (e == cudaSuccess) done = true;
    return e;
}
template <class T>
static cudaError_t push_batched_impl(int v, const void* args, const void* items, int n_items, cudaStream_t st) {
    const PushArgs<T>* a = (const PushArgs<T>*)args;
    const PushItem* it = (const PushItem*)items;
    if (v == 1)
        k_push_staged<T><<<(unsigned)n_items * (256 / PUSH_PPB), PUSH_PPB, push_staged_smem<T>(), st>>>(a, it);
    else if (v == PUSH_VARIANT_SUB)
        k_push_batched<T, 128, 3, true><<<(unsigned)n_items * 2, 128, 0, st>>>(a, it);
    else if (v == PUSH_VARIANT_RECORD)
        k_push_record<T, 128, 4><<<(unsigned)n_items * 2, 128, 0, st>>>(a, it);
    else if (v == PUSH_VARIANT_SPLIT) {
        k_push_force<T, 128, SPLIT_FORCE_MINB><<<(unsigned)n_items * 2, 128, 0, st>>>(a, it);
        k_push_move<T, 128, SPLIT_MOVE_MINB><<<(unsigned)n_items * 2, 128, 0, st>>>(a, it);
    }
    else
        k_push_batched<T, 128, 3><<<(unsigned)n_items * 2, 128, 0, st>>>(a, it);
    return cudaGetLastError();
}
cudaError_t launch_push_batched(int prec, int v, const void* args, const void* items, int n_items, cudaStream_t st) {
    if (n_items <= 0) return cudaSuccess;
    if (v < 0 || (v >= push_variants() && v != PUSH_VARIANT_SUB)) return cudaErrorInvalidValue;
    return prec ? push_batched_impl<float>(v, args, items, n_items, st)
                : push_batched_impl<double>(v, args, items, n_items, st);
}
// The push waits on scattered field loads (long-scoreboard stalls), so resident warps
// decide its speed.  With the stored plaquettes (no clover products) the FP32 push of the
// default path runs 4 blocks of 128 threads per SM (128 registers, 48 B of spills, 16
// warps): 1M sorted partons on 1024^2 in 310.5 instead of 328.3 us per coupled step at 3
// blocks (256-thread blocks, 8 warps, before the plaquettes: 414 us).  The FP32 sub-cycled /
// cloud-in-cell push stays at 3 blocks (168 registers): at 4 it spills 140 B and loses (87.8
// against 71.8 ms for 409 steps of 200k quarks on 512^2).  FP64 stays at 8 warps.
cudaError_t launch_push(int prec, const PushHost& a, const PartHost& P, cudaStream_t st) {
    if (a.np <= 0) return cudaSuccess;
    const int nb = (a.np + 255) / 256;
    if (a.nsub > 1 || a.interp) {
        if (prec) k_push<float, true, 128, 3><<<(a.np + 127) / 128, 128, 0, st>>>(push_args<float>(a, P));
        else k_push<double, true, 256, 1><<<nb, 256, 0, st>>>(push_args<double>(a, P));
    } else {
        if (prec) k_push<float, false, 128, 4><<<(a.np + 127) / 128, 128, 0, st>>>(push_args<float>(a, P));
        else k_push<double, false, 256, 1><<<nb, 256, 0, st>>>(push_args<double>(a, P));
    }
    return cudaGetLastError();
}

// Ensembles of one event pushed together (default path, no sub-steps, nearest grid
// point): one launch of 128-thread blocks, 4 per SM in FP32, the ensembles' blocks interleaved.
template <class T>
static cudaError_t push_pack_impl(const PushHost* a, const PartHost* const* P, int n, cudaStream_t st) {
    PushPack<T> pk;
    int nbmax = 0;
    for (int i = 0; i < n; i++) {
        pk.a[i] = push_args<T>(a[i], *P[i]);
        nbmax = std::max(nbmax, (a[i].np + 127) / 128);
    }
    pk.n = n;
    if (nbmax == 0) return cudaSuccess;
    if constexpr (std::is_same<T, float>::value) k_push_pack<T, 128, 4><<<nbmax * n, 128, 0, st>>>(pk);
    else k_push_pack<T, 128, 2><<<nbmax * n, 128, 0, st>>>(pk);
    return cudaGetLastError();
}
cudaError_t launch_push_pack(int prec, const PushHost* a, const PartHost* const* P, int n, cudaStream_t st) {
    if (n < 1 || n > PUSH_PACK) return cudaErrorInvalidValue;
    return prec ? push_pack_impl<float>(a, P, n, st) : push_pack_impl<double>(a, P, n, st);
}

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

size_t sort_scratch_ints(int ncell) { return 2 * (size_t)ncell + (size_t)(ncell + 1023) / 1024 + 1; }

cudaError_t launch_sort(int prec, const PartHost& a, const PartHost& b, int np, int ncell, int* count, int* start,
                        int* totals, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int) * ncell, st);
    if (e != cudaSuccess) return e;
    const int nbp = (np + 255) / 256;
    if (np > 0) k_cell_count<<<nbp, 256, 0, st>>>(a.cell, np, count);
    const int nbs = (ncell + 1023) / 1024;
    k_scan_block<<<nbs, 1024, 0, st>>>(count, start, totals, ncell);
    k_scan_totals<<<1, 32, 0, st>>>(totals, nbs);
    k_scan_add<<<nbs, 1024, 0, st>>>(start, totals, ncell);
    if (np > 0) {
        if (prec) k_scatter<float><<<nbp, 256, 0, st>>>(soa<float>(a), soa<float>(b), np, start);
        else k_scatter<double><<<nbp, 256, 0, st>>>(soa<double>(a), soa<double>(b), np, start);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- initial state
// Haar U(3) from 9 complex Gaussians: modified Gram-Schmidt of the columns
// (R has a positive diagonal, Mezzadri 2007)
DEV M3<double> haar(const double g[18]) {
    M3<double> Z, U;
    const double r2 = 0.70710678118654752440;
#pragma unroll
    for (int k = 0; k < 9; k++) Z.m[k / 3][k % 3] = mk(g[2 * k] * r2, g[2 * k + 1] * r2);
#pragma unroll
    for (int j = 0; j < 3; j++) {
        cx<double> v[3] = {Z.m[0][j], Z.m[1][j], Z.m[2][j]};
        for (int k = 0; k < j; k++) {
            cx<double> ip = mk(0.0, 0.0);
            for (int i = 0; i < 3; i++) fmca_(ip, U.m[i][k], v[i]);
            for (int i = 0; i < 3; i++) v[i] = v[i] - ip * U.m[i][k];
        }
        double nv = 0;
        for (int i = 0; i < 3; i++) nv += v[i].r * v[i].r + v[i].i * v[i].i;
        nv = 1.0 / sqrt(nv);
        for (int i = 0; i < 3; i++) U.m[i][j] = nv * v[i];
    }
    return U;
}

template <class T>
__global__ void k_part_init(PartSoA<T> P, int np, int n, int kind, double pmin, double pmax, double q3c,
                            double q8c, uint2 key) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= np) return;
    const uint4 r = philox4x32_10(make_uint4((uint32_t)j, 0u, 0u, 2u), key);
    const double x = n * u01(r.x), y = n * u01(r.y);
    const double pm = pmin + (pmax - pmin) * u01(r.z);
    double sa, ca;
    sincospi(2.0 * u01(r.w), &sa, &ca);
    double px, py;
    if (kind == 0) { px = pm * ca; py = pm * sa; }
    else { px = pm; py = 0.0; }
    double g[20];
#pragma unroll
    for (int k = 1; k <= 5; k++) {
        const uint4 q = philox4x32_10(make_uint4((uint32_t)j, 0u, (uint32_t)k, 2u), key);
        box_muller(q.x, q.y, g[4 * (k - 1)], g[4 * (k - 1) + 1]);
        box_muller(q.z, q.w, g[4 * (k - 1) + 2], g[4 * (k - 1) + 3]);
    }
    const M3<double> U = haar(g);
    Al<double> q0;
#pragma unroll
    for (int a = 0; a < 8; a++) q0.a[a] = 0.0;
    q0.a[2] = q3c;
    q0.a[7] = q8c;
    const Al<double> q = conj_alg(U, q0);
    const double fx = floor(x), fy = floor(y);
    int cx = (int)fx, cy = (int)fy;
    if (cx >= n) cx = n - 1;
    if (cy >= n) cy = n - 1;
    P.cell[j] = cx + n * cy;
    P.pid[j] = j;
    P.ox[j] = clamp_below_one((T)(x - fx));
    P.oy[j] = clamp_below_one((T)(y - fy));
    P.eta[j] = T(0);
    P.p0x[j] = (T)px;
    P.p0y[j] = (T)py;
    P.p0z[j] = T(0);
    P.dpx[j] = T(0);
    P.dpy[j] = T(0);
    P.peta[j] = T(0);
#pragma unroll
    for (int a = 0; a < 8; a++) P.Q[(size_t)a * P.qs + j] = (T)q.a[a];
}

// Cartan Q0 = Q3 t^3 + Q8 t^8 with Q3^2 + Q8^2 = q2 and (3 q2 Q8 - 4 Q8^3)/sqrt3 = q3:
// trigonometric roots of the depressed cubic, smallest positive one
static void cartan_q0(double q2, double q3, double* Q3, double* Q8) {
    const double p = -0.75 * q2, qq = sqrt(3.0) * q3 / 4.0;
    const double m = 2.0 * sqrt(-p / 3.0);
    double arg = (3.0 * qq / (2.0 * p)) * sqrt(-3.0 / p);
    arg = arg > 1 ? 1 : (arg < -1 ? -1 : arg);
    const double th = acos(arg) / 3.0;
    double best = 1e300;
    for (int k = 0; k < 3; k++) {
        const double r = m * cos(th - 2.0 * M_PI * k / 3.0);
        if (r > 0 && r < best) best = r;
    }
    *Q8 = best;
    *Q3 = sqrt(fmax(q2 - best * best, 0.0));
}

cudaError_t launch_part_init(int prec, const PartHost& P, int np, int n, int kind, double pmin, double pmax,
                             double q2, double q3, uint64_t seed, double mass, cudaStream_t st) {
    (void)mass;
    if (np <= 0) return cudaSuccess;
    double Q3, Q8;
    cartan_q0(q2, q3, &Q3, &Q8);
    const uint2 key = make_uint2((uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
    const int nb = (np + 127) / 128;
    if (prec) k_part_init<float><<<nb, 128, 0, st>>>(soa<float>(P), np, n, kind, pmin, pmax, Q3, Q8, key);
    else k_part_init<double><<<nb, 128, 0, st>>>(soa<double>(P), np, n, kind, pmin, pmax, Q3, Q8, key);
    return cudaGetLastError();
}

template <class T>
__global__ void k_part_from(PartSoA<T> P, int np, int n, const double* __restrict__ d) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= np) return;
    const double x = d[j], y = d[(size_t)np + j];
    const double fx = floor(x), fy = floor(y);
    int cx = ((int)fx % n + n) % n, cy = ((int)fy % n + n) % n;
    P.cell[j] = cx + n * cy;
    P.pid[j] = j;
    P.ox[j] = clamp_below_one((T)(x - fx));
    P.oy[j] = clamp_below_one((T)(y - fy));
    P.eta[j] = (T)d[2 * (size_t)np + j];
    const double px = d[3 * (size_t)np + j], py = d[4 * (size_t)np + j];
    const double p0x = d[14 * (size_t)np + j], p0y = d[15 * (size_t)np + j], p0z = d[16 * (size_t)np + j];
    P.p0x[j] = (T)p0x;
    P.p0y[j] = (T)p0y;
    P.p0z[j] = (T)p0z;
    P.dpx[j] = (T)(px - p0x);
    P.dpy[j] = (T)(py - p0y);
    P.peta[j] = (T)d[5 * (size_t)np + j];
#pragma unroll
    for (int a = 0; a < 8; a++) P.Q[(size_t)a * P.qs + j] = (T)d[(6 + a) * (size_t)np + j];
}
template <class T>
__global__ void k_part_to(PartSoA<T> P, int np, int n, double* __restrict__ d) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= np) return;
    const int k = P.pid[j];
    const int c = P.cell[j];
    d[k] = (double)(c % n) + (double)P.ox[j];
    d[(size_t)np + k] = (double)(c / n) + (double)P.oy[j];
    d[2 * (size_t)np + k] = (double)P.eta[j];
    d[3 * (size_t)np + k] = (double)P.p0x[j] + (double)P.dpx[j];
    d[4 * (size_t)np + k] = (double)P.p0y[j] + (double)P.dpy[j];
    d[5 * (size_t)np + k] = (double)P.peta[j];
#pragma unroll
    for (int a = 0; a < 8; a++) d[(6 + a) * (size_t)np + k] = (double)P.Q[(size_t)a * P.qs + j];
}
cudaError_t launch_part_from_canonical(int prec, const PartHost& P, int np, int n, const double* d, cudaStream_t st) {
    if (np <= 0) return cudaSuccess;
    const int nb = (np + 255) / 256;
    if (prec) k_part_from<float><<<nb, 256, 0, st>>>(soa<float>(P), np, n, d);
    else k_part_from<double><<<nb, 256, 0, st>>>(soa<double>(P), np, n, d);
    return cudaGetLastError();
}
cudaError_t launch_part_to_canonical(int prec, const PartHost& P, int np, int n, double* d, cudaStream_t st) {
    if (np <= 0) return cudaSuccess;
    const int nb = (np + 255) / 256;
    if (prec) k_part_to<float><<<nb, 256, 0, st>>>(soa<float>(P), np, n, d);
    else k_part_to<double><<<nb, 256, 0, st>>>(soa<double>(P), np, n, d);
    return cudaGetLastError();
}

template <class T>
__global__ void k_casimir(PartSoA<T> P, int np, double q2, double q3, double* out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    double d2 = 0, d3 = 0;
    if (j < np) {
        Al<double> q;
        for (int a = 0; a < 8; a++) q.a[a] = (double)P.Q[(size_t)a * P.qs + j];
        double s2 = 0;
        for (int a = 0; a < 8; a++) s2 += q.a[a] * q.a[a];
        // q3 = 4 Tr Q^3 = 4 sum_ij (Q^2)_ij Q_ji
        const H3<double> X = herm(q), X2 = hsq(X);
        double t = 0;
        for (int i = 0; i < 3; i++)
            for (int k = 0; k < 3; k++) {
                const cx<double> a = hget(X2, i, k), b = hget(X, k, i);
                t += a.r * b.r - a.i * b.i;
            }
        d2 = fabs(s2 - q2);
        d3 = fabs(4.0 * t - q3);
    }
    for (int o = 16; o > 0; o >>= 1) {
        d2 = fmax(d2, __shfl_down_sync(0xffffffffu, d2, o));
        d3 = fmax(d3, __shfl_down_sync(0xffffffffu, d3, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(reinterpret_cast<unsigned long long*>(out), (unsigned long long)__double_as_longlong(d2));
        atomicMax(reinterpret_cast<unsigned long long*>(out + 1), (unsigned long long)__double_as_longlong(d3));
    }
}
cudaError_t launch_casimir_drift(int prec, const PartHost& P, int np, double q2, double q3, double* out2,
                                 cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out2, 0, 2 * sizeof(double), st);
    if (e != cudaSuccess || np <= 0) return e;
    const int nb = (np + 255) / 256;
    if (prec) k_casimir<float><<<nb, 256, 0, st>>>(soa<float>(P), np, q2, q3, out2);
    else k_casimir<double><<<nb, 256, 0, st>>>(soa<double>(P), np, q2, q3, out2);
    return cudaGetLastError();
}

}  // namespace glasma
