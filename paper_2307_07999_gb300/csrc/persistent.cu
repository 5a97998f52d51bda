// Persistent batched kernel: one cooperative launch advances every event of a
// batch through its whole evolution (the coupled field + particle steps of
// Sec. 1 of arXiv:2307.07999 for all events of the Sec. 2 event average).
//
// Phase p runs the field tiles of iteration p and the particle blocks of
// iteration p-1.  The tiles are dealt out statically (CTA b takes tiles b,
// b + grid, ...: equal shares, no atomic per tile); then each CTA takes particle
// blocks from an atomic work counter, so the CTAs that finish their tiles first
// push while the others still step fields.  The three rotating field buffers keep
// the two apart: iteration p reads buf[p%3] and writes buf[(p+1)%3]; the push of
// iteration p-1 reads buf[(p-1)%3] and buf[p%3].
// Phases are separated by a grid barrier whose wait is bounded: when it runs out
// the kernel raises an error word and returns, and the host reports
// GLASMA_ERR_TIMEOUT.  Field and particle loads go through L2 (ld.global.cg)
// because the kernel reads in later phases what other CTAs wrote earlier.
#include <stdio.h>

#include <algorithm>

#include "batch.h"
#include "particles.cuh"

namespace glasma {

struct PersCtl {
    unsigned count;
    unsigned gen;
    int err;
};

template <class T> struct PersArgs {
    const StepArgs<T>* sargs;  // [K][E]
    const PushArgs<T>* pargs;  // [K][E]
    const TileItem* tiles;
    const PushItem* pitems;
    PersCtl* ctl;
    int* work;                 // [K + 1]
    const int* active;         // [K]
    const int* tiles_upto;     // [E + 1]
    const int* pitems_upto;    // [E + 1]
    int E, K;
    unsigned long long spin_limit;
};

// Three CTAs of 128 threads per SM (168 registers, 12 warps): 482 ms for the 64-event
// batch against 552 at two CTAs (255 registers, 8 warps).
#ifndef GLASMA_PERS_MINB
#define GLASMA_PERS_MINB 3
#endif
template <class T> struct PersCfg { static constexpr int TX = 32, TY = 4, MINB = GLASMA_PERS_MINB; };
template <> struct PersCfg<double> { static constexpr int TX = 32, TY = 4, MINB = 1; };

// all CTAs arrive; false if the wait ran out (then the error word is set)
DEV bool grid_barrier(PersCtl* c, unsigned nblocks, unsigned long long limit) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        int good = 1;
        volatile unsigned* gen = &c->gen;
        const unsigned g = *gen;
        __threadfence();
        if (atomicAdd(&c->count, 1u) == nblocks - 1) {
            atomicExch(&c->count, 0u);
            __threadfence();
            atomicAdd(&c->gen, 1u);
        } else {
            unsigned long long it = 0;
            while (*gen == g) {
                if (++it > limit) {
                    atomicExch(&c->err, 1);
                    good = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        if (*(volatile int*)&c->err) good = 0;
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

template <class T>
__global__ void __launch_bounds__(PersCfg<T>::TX * PersCfg<T>::TY, PersCfg<T>::MINB)
k_persistent(PersArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int TX = PersCfg<T>::TX, TY = PersCfg<T>::TY, NT = TX * TY;
    __shared__ int s_item;
    const int tid = threadIdx.y * TX + threadIdx.x;
    for (int p = 0; p <= a.K; p++) {
        const int actF = p < a.K ? a.active[p] : 0;       // events advancing their fields at iteration p
        const int actP = p >= 1 ? a.active[p - 1] : 0;    // events pushing at iteration p-1
        const int nt = actF ? a.tiles_upto[actF] : 0;
        const int npi = actP ? a.pitems_upto[actP] : 0;
        for (int i = blockIdx.x; i < nt; i += gridDim.x) {
            const TileItem ti = a.tiles[i];
            field_tile<T, TX, TY, true>(a.sargs[(size_t)p * a.E + ti.ev], ti.x0, ti.y0, smem);
            __syncthreads();
        }
        for (;;) {
            if (tid == 0) s_item = atomicAdd(a.work + p, 1);
            __syncthreads();
            const int i = s_item;
            __syncthreads();
            if (i >= npi) break;
            {
                const PushItem it = a.pitems[i];
                const PushArgs<T>& A = a.pargs[(size_t)(p - 1) * a.E + it.ev];
                if (A.acc != nullptr) {
                    double sx = 0.0, sy = 0.0, sz = 0.0, sc = 0.0;
                    for (int h = 0; h < 256 / NT; h++) {
                        const int j = it.j0 + h * NT + tid;
                        if (j < A.np) {
                            T a0, a1, a2, a3;
                            push_one<T, true>(A, j, a0, a1, a2, a3);
                            sx += a0; sy += a1; sz += a2; sc += a3;
                        }
                    }
                    block_acc4(sx, sy, sz, sc, A.acc);
                    __syncthreads();
                }
            }
        }
        if (!grid_barrier(a.ctl, gridDim.x, a.spin_limit)) return;
    }
}

template <class T> static glasma_status run_impl(glasma_batch* b) {
    constexpr int TX = PersCfg<T>::TX, TY = PersCfg<T>::TY;
    const size_t sm = RecTile<T, TX, TY>::smem;
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_persistent<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
            return GLASMA_ERR_CUDA;
        attr = true;
    }
    if (b->pers_blocks == 0) {
        int dev = 0, sms = 0, per = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_persistent<T>, TX * TY, sm) != cudaSuccess || per < 1)
            return GLASMA_ERR_CUDA;
        b->pers_blocks = sms * per;
    }
    const int K = std::max(1, b->max_iter), E = b->E;
    char* base = (char*)b->pers_ctrl;
    int* ints = (int*)(base + 256);
    PersArgs<T> a;
    a.sargs = (const StepArgs<T>*)b->step_args;
    a.pargs = (const PushArgs<T>*)b->push_args;
    a.tiles = (const TileItem*)b->tiles_dev;
    a.pitems = (const PushItem*)b->pitems_dev;
    a.ctl = (PersCtl*)base;
    a.work = ints;
    a.active = ints + (K + 1);
    a.tiles_upto = ints + (K + 1) + K;
    a.pitems_upto = ints + (K + 1) + K + (E + 1);
    a.E = E;
    a.K = b->max_iter;
    a.spin_limit = b->pers_spin;  // default 2^24 polls: ~2 s at ~100 ns per poll
    if (cudaMemsetAsync(base, 0, 256 + (size_t)(K + 1) * 4, b->st) != cudaSuccess) return GLASMA_ERR_CUDA;
    void* args[] = {&a};
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_persistent<T>, dim3(b->pers_blocks), dim3(TX, TY), args,
                                                sm, b->st);
    if (e == cudaSuccess) b->pers_launched = true;
    return e == cudaSuccess ? GLASMA_OK : GLASMA_ERR_CUDA;
}

}  // namespace glasma

using namespace glasma;

static cudaError_t restore_all(glasma_batch* b) {
    for (auto& x : b->ev) {
        const size_t fb = align256((size_t)N_FIELD_PLANES * x.ns * (b->prec ? 4 : 8));
        cudaError_t e = cudaMemcpyAsync(x.buf[0], x.init_buf, fb, cudaMemcpyDeviceToDevice, b->st);
        if (e != cudaSuccess) return e;
        e = cudaMemcpyAsync(x.part_base, x.part_init, x.part_bytes, cudaMemcpyDeviceToDevice, b->st);
        if (e != cudaSuccess) return e;
        e = cudaMemsetAsync(x.acc, 0, (size_t)x.acc_rows * 4 * 8, b->st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

glasma_status batch_run_persistent(glasma_batch* b) {
    if (restore_all(b) != cudaSuccess) {
        glasma_set_error("persistent run: restore failed");
        return GLASMA_ERR_CUDA;
    }
    const glasma_status s = b->prec ? run_impl<float>(b) : run_impl<double>(b);
    if (s != GLASMA_OK) glasma_set_error(cudaGetErrorString(cudaGetLastError()));
    return s;
}

bool batch_timed_out(glasma_batch* b) {
    if (!b->pers_ctrl || !b->pers_launched) return false;
    int err = 0;
    if (cudaMemcpy(&err, (char*)b->pers_ctrl + 8, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return false;
    if (err) cudaMemset((char*)b->pers_ctrl + 8, 0, sizeof(int));
    return err != 0;
}

void batch_free_persistent(glasma_batch* b) { (void)b; }

extern "C" glasma_status glasma_batch_set_wait_limit(glasma_batch* b, int64_t polls) {
    if (!b || polls < 0 || polls > (int64_t(1) << 40)) {
        glasma_set_error("glasma_batch_set_wait_limit: bad arguments");
        return GLASMA_ERR_INVALID;
    }
    b->pers_spin = polls == 0 ? (1ull << 24) : (unsigned long long)polls;
    return GLASMA_OK;
}
