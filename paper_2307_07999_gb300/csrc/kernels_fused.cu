// Batched fused field step + particle push (one CTA per event tile), and the
// per-step binning of particle indices by tile that feeds it.
#include "fused.cuh"
#include "internal.h"

namespace glasma {

#ifndef GLASMA_FUSED_MINB
#define GLASMA_FUSED_MINB 2
#endif
template <class T> struct FusedCfg { static constexpr int TX = 32, TY = 4, MINB = GLASMA_FUSED_MINB; };
template <> struct FusedCfg<double> { static constexpr int TX = 32, TY = 4, MINB = 1; };

template <class T>
__global__ void __launch_bounds__(FusedCfg<T>::TX * FusedCfg<T>::TY, FusedCfg<T>::MINB)
k_fused_batched(const StepArgs<T>* __restrict__ args, const PushArgs<T>* __restrict__ pargs,
                const TileItem* __restrict__ items, const int* __restrict__ start, const int* __restrict__ count,
                const int* __restrict__ perm) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int TX = FusedCfg<T>::TX, TY = FusedCfg<T>::TY;
    const TileItem it = items[blockIdx.x];
    fused_tile<T, TX, TY>(args[it.ev], pargs[it.ev], it.x0, it.y0, perm, start[blockIdx.x], count[blockIdx.x], smem);
}

int fused_tile_x(int prec) { return prec ? FusedCfg<float>::TX : FusedCfg<double>::TX; }
int fused_tile_y(int prec) { return prec ? FusedCfg<float>::TY : FusedCfg<double>::TY; }

template <class T> static cudaError_t fused_impl(const void* args, const void* pargs, const void* items, int n_items,
                                                 const int* start, const int* count, const int* perm, cudaStream_t st) {
    constexpr int TX = FusedCfg<T>::TX, TY = FusedCfg<T>::TY;
    const size_t sm = FusedTile<T, TX, TY>::smem;
    static bool done = false;
    if (!done) {
        cudaError_t e = cudaFuncSetAttribute(k_fused_batched<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        done = true;
    }
    if (n_items <= 0 || !args) return cudaSuccess;
    k_fused_batched<T><<<n_items, dim3(TX, TY), sm, st>>>((const StepArgs<T>*)args, (const PushArgs<T>*)pargs,
                                                         (const TileItem*)items, start, count, perm);
    return cudaGetLastError();
}
cudaError_t launch_fused_batched(int prec, const void* args, const void* pargs, const void* items, int n_items,
                                 const int* start, const int* count, const int* perm, cudaStream_t st) {
    return prec ? fused_impl<float>(args, pargs, items, n_items, start, count, perm, st)
                : fused_impl<double>(args, pargs, items, n_items, start, count, perm, st);
}

// ---------------------------------------------------------------- binning by tile
// event e's particle j sits in tile (cy / TY) * ntx + cx / TX of that event; tiles of
// all events are numbered consecutively (tile_base)
__global__ void k_tile_count(const BinArgs* __restrict__ bins, const PushItemH* __restrict__ items,
                             int* __restrict__ count) {
    const PushItemH it = items[blockIdx.x];
    const BinArgs b = bins[it.ev];
    const int j = it.j0 + threadIdx.x;
    if (j >= b.np) return;
    const int c = b.cell[j];
    const int cx = c % b.n, cy = c / b.n;
    atomicAdd(count + b.tile_base + (cy / b.ty) * b.ntx + cx / b.tx, 1);
}
__global__ void k_tile_scatter(const BinArgs* __restrict__ bins, const PushItemH* __restrict__ items,
                               const int* __restrict__ start, int* __restrict__ fill, int* __restrict__ perm) {
    const PushItemH it = items[blockIdx.x];
    const BinArgs b = bins[it.ev];
    const int j = it.j0 + threadIdx.x;
    if (j >= b.np) return;
    const int c = b.cell[j];
    const int cx = c % b.n, cy = c / b.n;
    const int t = b.tile_base + (cy / b.ty) * b.ntx + cx / b.tx;
    perm[start[t] + atomicAdd(fill + t, 1)] = j;
}

// exclusive scan of count into start (three passes, 1024 per block)
__global__ void k_bscan_block(const int* __restrict__ in, int* __restrict__ out, int* __restrict__ totals, int len) {
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
__global__ void k_bscan_totals(int* totals, int nb) {
    __shared__ int buf[1024];
    // nb <= 1024 * 1024 tiles / 1024 = 1024 blocks: one block scans them
    int run = 0;
    for (int base = 0; base < nb; base += 1024) {
        const int i = base + threadIdx.x;
        const int v = i < nb ? totals[i] : 0;
        buf[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            const int t = threadIdx.x >= o ? buf[threadIdx.x - o] : 0;
            __syncthreads();
            buf[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < nb) totals[i] = run + buf[threadIdx.x] - v;
        run += buf[1023];
        __syncthreads();
    }
}
__global__ void k_bscan_add(int* __restrict__ out, const int* __restrict__ totals, int len) {
    const int i = blockIdx.x * 1024 + threadIdx.x;
    if (i < len) out[i] += totals[blockIdx.x];
}

cudaError_t launch_rebin(const void* bins, const void* pitems, int n_pitems, int n_tiles, int* count, int* fill,
                         int* start, int* totals, int* perm, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int) * (size_t)n_tiles, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(fill, 0, sizeof(int) * (size_t)n_tiles, st);
    if (e != cudaSuccess) return e;
    if (n_pitems > 0) k_tile_count<<<n_pitems, 256, 0, st>>>((const BinArgs*)bins, (const PushItemH*)pitems, count);
    const int nb = (n_tiles + 1023) / 1024;
    k_bscan_block<<<nb, 1024, 0, st>>>(count, start, totals, n_tiles);
    k_bscan_totals<<<1, 1024, 0, st>>>(totals, nb);
    k_bscan_add<<<nb, 1024, 0, st>>>(start, totals, n_tiles);
    if (n_pitems > 0)
        k_tile_scatter<<<n_pitems, 256, 0, st>>>((const BinArgs*)bins, (const PushItemH*)pitems, start, fill, perm);
    return cudaGetLastError();
}

}  // namespace glasma
