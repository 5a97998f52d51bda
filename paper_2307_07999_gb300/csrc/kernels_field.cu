// Field kernels: fused kick+drift step (single event and batched over events),
// canonical-layout conversion and FP64 monitors (Gauss law, energy densities,
// unitarity).  Physics: Sec. 1 ("Glasma") of arXiv:2307.07999.
#include "field.cuh"
#include "internal.h"

namespace glasma {

#ifndef GLASMA_FIELD_TY
#define GLASMA_FIELD_TY 4
#endif
#ifndef GLASMA_FIELD_MINB
#define GLASMA_FIELD_MINB 3
#endif
template <class T> struct TileCfg;
template <> struct TileCfg<float> { static constexpr int TX = 32, TY = GLASMA_FIELD_TY, MINB = GLASMA_FIELD_MINB; };
template <> struct TileCfg<double> { static constexpr int TX = 32, TY = 4, MINB = 1; };

template <class T>
__global__ void __launch_bounds__(TileCfg<T>::TX * TileCfg<T>::TY, TileCfg<T>::MINB)
k_field_step(StepArgs<T> A) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int TX = TileCfg<T>::TX, TY = TileCfg<T>::TY;
    field_tile<T, TX, TY, false, false, true>(A, blockIdx.x * TX, blockIdx.y * TY, smem);
}
template <class T, bool REC = false>
__global__ void __launch_bounds__(TileCfg<T>::TX * TileCfg<T>::TY, TileCfg<T>::MINB)
k_field_step_batched(const StepArgs<T>* __restrict__ args, const TileItem* __restrict__ items) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int TX = TileCfg<T>::TX, TY = TileCfg<T>::TY;
    const TileItem it = items[blockIdx.x];
    field_tile<T, TX, TY, false, REC>(args[it.ev], it.x0, it.y0, smem);
}

StepHost step_coeffs(const void* src, void* dst, int n, int step, double dtau, int expanding, int reunit) {
    StepHost a;
    a.src = src; a.dst = dst; a.n = n; a.dtau = dtau; a.reunit = reunit;
    a.plaq = const_cast<void*>(src);  // the plaquettes of src's links go into src's last group
    a.rec = nullptr; a.occ = nullptr; a.epoch = step; a.all_rec = 0;
    const double tn = step * dtau, th = (step + 0.5) * dtau;
    a.tb = expanding ? tn : 1.0;
    a.tp = expanding ? 1.0 / tn : 1.0;
    a.ue = expanding ? dtau / th : dtau;
    a.pe = expanding ? dtau * th : dtau;
    return a;
}

template <class T> static StepArgs<T> to_args(const StepHost& a) {
    StepArgs<T> A;
    A.src = (const T*)a.src; A.dst = (T*)a.dst; A.n = a.n;
    A.tb = (T)a.tb; A.tp = (T)a.tp; A.dtau = (T)a.dtau; A.ue = (T)a.ue; A.pe = (T)a.pe;
    A.reunit = a.reunit;
    A.plaq = (T*)a.plaq;
    A.rec = (T*)a.rec; A.occ = a.occ; A.epoch = a.epoch; A.all_rec = a.all_rec;
    return A;
}
size_t step_args_size(int prec) { return prec ? sizeof(StepArgs<float>) : sizeof(StepArgs<double>); }
void pack_step_args(int prec, const StepHost& a, void* out) {
    if (prec) *(StepArgs<float>*)out = to_args<float>(a);
    else *(StepArgs<double>*)out = to_args<double>(a);
}
int field_tile_x(int prec) { return prec ? TileCfg<float>::TX : TileCfg<double>::TX; }
int field_tile_y(int prec) { return prec ? TileCfg<float>::TY : TileCfg<double>::TY; }

template <class T> static cudaError_t set_smem() {
    constexpr int TX = TileCfg<T>::TX, TY = TileCfg<T>::TY;
    const size_t sm = RecTile<T, TX, TY>::smem;
    static bool done = false;
    if (!done) {
        cudaError_t e = cudaFuncSetAttribute(k_field_step<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_field_step_batched<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_field_step_batched<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        done = true;
    }
    return cudaSuccess;
}

// single-event FP32 step in a tile shape the batch tuner picks on the 64-event batch of
// 128^2-512^2 lattices
// (16 x 8 sites, 4 CTAs per SM); the per-site arithmetic is that of every shape
template <int TX, int TY, int MINB>
__global__ void __launch_bounds__(TX * TY, MINB) k_field_step_grid(StepArgs<float> A) {
    extern __shared__ __align__(16) unsigned char smem[];
    field_tile<float, TX, TY, false, false, true>(A, blockIdx.x * TX, blockIdx.y * TY, smem);
}
constexpr int SINGLE_TX = 16, SINGLE_TY = 8, SINGLE_MINB = 4;

template <class T> static cudaError_t step_impl(const StepHost& a, cudaStream_t st) {
    constexpr int TX = TileCfg<T>::TX, TY = TileCfg<T>::TY;
    cudaError_t e = set_smem<T>();
    if (e != cudaSuccess) return e;
    dim3 grid((a.n + TX - 1) / TX, (a.n + TY - 1) / TY), block(TX, TY);
    k_field_step<T><<<grid, block, RecTile<T, TX, TY>::smem, st>>>(to_args<T>(a));
    return cudaGetLastError();
}
template <> cudaError_t step_impl<float>(const StepHost& a, cudaStream_t st) {
    constexpr int TX = SINGLE_TX, TY = SINGLE_TY;
    constexpr size_t sm = RecTile<float, TX, TY>::smem;
    static bool done = false;
    if (!done) {
        cudaError_t e = cudaFuncSetAttribute(k_field_step_grid<TX, TY, SINGLE_MINB>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        done = true;
    }
    dim3 grid((a.n + TX - 1) / TX, (a.n + TY - 1) / TY), block(TX, TY);
    k_field_step_grid<TX, TY, SINGLE_MINB><<<grid, block, sm, st>>>(to_args<float>(a));
    return cudaGetLastError();
}
cudaError_t launch_field_step(int prec, const StepHost& a, cudaStream_t st) {
    return prec ? step_impl<float>(a, st) : step_impl<double>(a, st);
}
template <class T>
static cudaError_t batched_impl(const void* args, const void* items, int n_items, bool rec, cudaStream_t st) {
    constexpr int TX = TileCfg<T>::TX, TY = TileCfg<T>::TY;
    cudaError_t e = set_smem<T>();
    if (e != cudaSuccess) return e;
    if (n_items <= 0 || !args) return cudaSuccess;
    const size_t sm = RecTile<T, TX, TY>::smem;
    if (rec)
        k_field_step_batched<T, true><<<n_items, dim3(TX, TY), sm, st>>>((const StepArgs<T>*)args,
                                                                          (const TileItem*)items);
    else
        k_field_step_batched<T><<<n_items, dim3(TX, TY), sm, st>>>((const StepArgs<T>*)args, (const TileItem*)items);
    return cudaGetLastError();
}
cudaError_t launch_field_step_batched(int prec, const void* args, const void* items, int n_items, cudaStream_t st,
                                      bool rec) {
    return prec ? batched_impl<float>(args, items, n_items, rec, st)
                : batched_impl<double>(args, items, n_items, rec, st);
}

// ---------------------------------------------------------------- FP32 tile variants
// The batched FP32 field step compiled for several tile shapes; a batch picks one by
// timing them on its own events (glasma_batch_tune).  The arithmetic per site is the
// same in every shape, so the results are identical.
template <int TX, int TY, int MINB, bool REC = false>
__global__ void __launch_bounds__(TX * TY, MINB)
k_field_step_tiles(const StepArgs<float>* __restrict__ args, const TileItem* __restrict__ items) {
    extern __shared__ __align__(16) unsigned char smem[];
    const TileItem it = items[blockIdx.x];
    field_tile<float, TX, TY, false, REC>(args[it.ev], it.x0, it.y0, smem);
}
struct FieldVariant {
    int tx, ty, minb;
    const void* fn;
    size_t smem;
    const void* fn_rec;  // the same shape writing the gather records
};
#define GL_FV(TX, TY, MB)                                                                                \
    {TX, TY, MB, (const void*)k_field_step_tiles<TX, TY, MB>, RecTile<float, TX, TY>::smem,             \
     (const void*)k_field_step_tiles<TX, TY, MB, true>}
static const FieldVariant g_fvar[] = {GL_FV(32, 4, 3), GL_FV(16, 8, 3), GL_FV(8, 16, 3), GL_FV(32, 6, 2),
                                      GL_FV(16, 12, 2), GL_FV(32, 8, 2), GL_FV(32, 4, 4), GL_FV(16, 8, 4),
                                      GL_FV(8, 8, 8), GL_FV(8, 16, 4), GL_FV(16, 16, 2)};
#undef GL_FV
static constexpr int N_FVAR = (int)(sizeof(g_fvar) / sizeof(g_fvar[0]));

int field_variants(int prec) { return prec ? N_FVAR : 1; }
void field_variant_shape(int prec, int v, int* tx, int* ty, int* minb) {
    if (!prec) { *tx = TileCfg<double>::TX; *ty = TileCfg<double>::TY; *minb = TileCfg<double>::MINB; return; }
    *tx = g_fvar[v].tx; *ty = g_fvar[v].ty; *minb = g_fvar[v].minb;
}
// shared-memory limits of every variant (call outside stream capture)
cudaError_t prepare_field_variants(int prec) {
    if (!prec) return set_smem<double>();
    cudaError_t e = set_smem<float>();
    static bool done = false;
    if (e != cudaSuccess || done) return e;
    for (int v = 0; v < N_FVAR; v++) {
        e = cudaFuncSetAttribute(g_fvar[v].fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g_fvar[v].smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(g_fvar[v].fn_rec, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g_fvar[v].smem);
        if (e != cudaSuccess) return e;
    }
    done = true;
    return cudaSuccess;
}
cudaError_t launch_field_step_variant(int prec, int v, const void* args, const void* items, int n_items,
                                      cudaStream_t st, bool rec) {
    if (!prec) return launch_field_step_batched(prec, args, items, n_items, st, rec);
    if (v < 0 || v >= N_FVAR) return cudaErrorInvalidValue;
    if (n_items <= 0 || !args) return cudaSuccess;
    const FieldVariant& f = g_fvar[v];
    void* kargs[2] = {(void*)&args, (void*)&items};
    return cudaLaunchKernel(rec ? f.fn_rec : f.fn, dim3((unsigned)n_items), dim3(f.tx, f.ty), kargs, f.smem, st);
}

// ---------------------------------------------------------------- canonical layout
template <class T>
__global__ void k_from_canonical(const double* __restrict__ U, const double* __restrict__ E,
                                 const double* __restrict__ phi, const double* __restrict__ pi, T* __restrict__ f,
                                 int n) {
    const size_t ns = (size_t)n * n;
    const size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (s >= ns) return;
#pragma unroll
    for (int d = 0; d < 2; d++)
#pragma unroll
        for (int k = 0; k < 12; k++)  // rows 0,1: entries 0..5, re/im
            f[fidx(12 * d + k, s, ns)] = (T)U[s * 36 + 18 * d + k];
#pragma unroll
    for (int a = 0; a < 16; a++) f[fidx(P_EX + a, s, ns)] = (T)E[s * 16 + a];
#pragma unroll
    for (int a = 0; a < 8; a++) {
        f[fidx(P_PHI + a, s, ns)] = (T)phi[s * 8 + a];
        f[fidx(P_PI + a, s, ns)] = (T)pi[s * 8 + a];
    }
}
template <class T>
__global__ void k_to_canonical(const T* __restrict__ f, double* __restrict__ U, double* __restrict__ E,
                               double* __restrict__ phi, double* __restrict__ pi, int n) {
    const size_t ns = (size_t)n * n;
    const size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (s >= ns) return;
    if (U) {
#pragma unroll
        for (int d = 0; d < 2; d++) {
            const M3<T> L = load_link(f, ns, d == 0 ? P_UX : P_UY, s);
#pragma unroll
            for (int k = 0; k < 9; k++) {
                U[s * 36 + 18 * d + 2 * k] = (double)L.m[k / 3][k % 3].r;
                U[s * 36 + 18 * d + 2 * k + 1] = (double)L.m[k / 3][k % 3].i;
            }
        }
    }
    if (E) {
#pragma unroll
        for (int a = 0; a < 16; a++) E[s * 16 + a] = (double)f[fidx(P_EX + a, s, ns)];
    }
    if (phi) {
#pragma unroll
        for (int a = 0; a < 8; a++) phi[s * 8 + a] = (double)f[fidx(P_PHI + a, s, ns)];
    }
    if (pi) {
#pragma unroll
        for (int a = 0; a < 8; a++) pi[s * 8 + a] = (double)f[fidx(P_PI + a, s, ns)];
    }
}
cudaError_t launch_state_from_canonical(int prec, const double* U, const double* E, const double* phi,
                                        const double* pi, void* buf, int n, cudaStream_t st) {
    const size_t ns = (size_t)n * n;
    const int nb = (int)((ns + 255) / 256);
    if (prec) k_from_canonical<float><<<nb, 256, 0, st>>>(U, E, phi, pi, (float*)buf, n);
    else k_from_canonical<double><<<nb, 256, 0, st>>>(U, E, phi, pi, (double*)buf, n);
    return cudaGetLastError();
}
cudaError_t launch_state_to_canonical(int prec, const void* buf, double* U, double* E, double* phi, double* pi,
                                      int n, cudaStream_t st) {
    const size_t ns = (size_t)n * n;
    const int nb = (int)((ns + 255) / 256);
    if (prec) k_to_canonical<float><<<nb, 256, 0, st>>>((const float*)buf, U, E, phi, pi, n);
    else k_to_canonical<double><<<nb, 256, 0, st>>>((const double*)buf, U, E, phi, pi, n);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- monitors (FP64 sums)
DEV void block_add(double v, double* dst) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(dst, v);
}
DEV void atomic_max_nonneg(double* dst, double v) {
    // non-negative doubles order like their bit patterns
    atomicMax(reinterpret_cast<unsigned long long*>(dst), (unsigned long long)__double_as_longlong(v));
}
template <class T>
__global__ void k_monitors(const T* __restrict__ f, int n, double te, double* mon) {
    const size_t ns = (size_t)n * n;
    const size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    double g2 = 0, den = 0, eet = 0, ebt = 0, eel = 0, ebl = 0, bad = 0, ud = 0;
    if (s < ns) {
        const int x = (int)(s % n), y = (int)(s / n);
        const size_t sxm = (x == 0 ? n - 1 : x - 1) + (size_t)n * y, sym = x + (size_t)n * (y == 0 ? n - 1 : y - 1);
        const size_t sxp = (x == n - 1 ? 0 : x + 1) + (size_t)n * y, syp = x + (size_t)n * (y == n - 1 ? 0 : y + 1);
        M3<T> ux, uy;
        load_links(f, ns, s, ux, uy);
        const Al<T> ex = load_alg(f, ns, P_EX, s), ey = load_alg(f, ns, P_EY, s);
        const Al<T> phi = load_alg(f, ns, P_PHI, s), pi = load_alg(f, ns, P_PI, s);
        // Gauss law G = sum_i [E_i(x) - U_i(x-i)^dag E_i(x-i) U_i(x-i)] + i[phi, pi]
        const Al<T> tx = transport_alg(load_link(f, ns, P_UX, sxm), load_alg(f, ns, P_EX, sxm));
        const Al<T> ty = transport_alg(load_link(f, ns, P_UY, sym), load_alg(f, ns, P_EY, sym));
        const Al<T> cm = icomm(phi, pi);
        double p2 = 0, q2 = 0;
        for (int a = 0; a < 8; a++) {
            const double g = (double)ex.a[a] + ey.a[a] - tx.a[a] - ty.a[a] + cm.a[a];
            g2 += g * g;
            den += 2.0 * ((double)ex.a[a] * ex.a[a] + (double)ey.a[a] * ey.a[a]);
            p2 += (double)phi.a[a] * phi.a[a];
            q2 += (double)pi.a[a] * pi.a[a];
            eet += 0.5 * ((double)ex.a[a] * ex.a[a] + (double)ey.a[a] * ey.a[a]);
            eel += 0.5 * (double)pi.a[a] * pi.a[a];
        }
        den += p2 * q2;
        const M3<T> P = mul_nd(mul(ux, load_link(f, ns, P_UY, sxp)), mul(uy, load_link(f, ns, P_UX, syp)));
        ebl = 2.0 * (3.0 - ((double)P.m[0][0].r + P.m[1][1].r + P.m[2][2].r));
        const Al<T> psx = conj_alg(ux, load_alg(f, ns, P_PHI, sxp));
        const Al<T> psy = conj_alg(uy, load_alg(f, ns, P_PHI, syp));
        for (int a = 0; a < 8; a++) {
            const double dx = (double)psx.a[a] - phi.a[a], dy = (double)psy.a[a] - phi.a[a];
            ebt += 0.5 * (dx * dx + dy * dy);
        }
        eet /= te * te;
        ebt /= te * te;
        const double tot = g2 + den + eet + ebt + eel + ebl;
        bad = isfinite(tot) ? 0.0 : 1.0;
        // rows 0,1 orthonormal (row 2 is their completion)
        for (int d = 0; d < 2; d++) {
            const M3<T>& U = d == 0 ? ux : uy;
            double n0 = 0, n1 = 0, ir = 0, ii = 0;
            for (int k = 0; k < 3; k++) {
                n0 += (double)U.m[0][k].r * U.m[0][k].r + (double)U.m[0][k].i * U.m[0][k].i;
                n1 += (double)U.m[1][k].r * U.m[1][k].r + (double)U.m[1][k].i * U.m[1][k].i;
                ir += (double)U.m[0][k].r * U.m[1][k].r + (double)U.m[0][k].i * U.m[1][k].i;
                ii += (double)U.m[0][k].r * U.m[1][k].i - (double)U.m[0][k].i * U.m[1][k].r;
            }
            ud = fmax(ud, fmax(fabs(n0 - 1.0), fmax(fabs(n1 - 1.0), sqrt(ir * ir + ii * ii))));
        }
    }
    block_add(g2, mon + 0);
    block_add(den, mon + 1);
    block_add(eet, mon + 2);
    block_add(ebt, mon + 3);
    block_add(eel, mon + 4);
    block_add(ebl, mon + 5);
    block_add(bad, mon + 7);
    for (int o = 16; o > 0; o >>= 1) ud = fmax(ud, __shfl_down_sync(0xffffffffu, ud, o));
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(mon + 6, ud);
}
cudaError_t launch_monitors(int prec, const void* buf, int n, double te, double* mon, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(mon, 0, 8 * sizeof(double), st);
    if (e != cudaSuccess) return e;
    const size_t ns = (size_t)n * n;
    const int nb = (int)((ns + 255) / 256);
    if (prec) k_monitors<float><<<nb, 256, 0, st>>>((const float*)buf, n, te, mon);
    else k_monitors<double><<<nb, 256, 0, st>>>((const double*)buf, n, te, mon);
    return cudaGetLastError();
}

}  // namespace glasma
