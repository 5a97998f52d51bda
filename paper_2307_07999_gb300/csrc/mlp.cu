// Learned warm start for the tau = 0+ link solve: a 36 -> 128 -> 128 -> 16 tanh
// network with BF16 weights and FP32 accumulation, trained on pairs that the
// method's own Newton solve produces.  (The paper has no learned component; the
// network only proposes a starting point, and the Newton iteration of the
// boost-invariant matching condition still decides the links to 1e-12.)
//
//   x = (a1, a2, c, d_s + c/2, |a1|^2, |a2|^2, a1.a2, |c|^2) / x_scale   36 inputs
//       a_k = im_tl(U_k), c = i[a1, a2], d_s the third-order series of ic.cuh
//   h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2), y = W3 h2 + b3   16 outputs
//   outputs 0..7: d_net / y_scale, the start being U0 = exp(i (d_s + d_net).t) U1 U2;
//   8..15: zero-target padding.  Training target: d - d_s, d the Newton solution's
//   offset 2 Im Tr[t^a U (U1 U2)^dag].
//
// Forward and backward activation products run on the tensor cores
// (mma.sync m16n8k16, BF16 operands, FP32 accumulators; a layer's FP32
// accumulator fragments are repacked in registers as the next layer's BF16
// operand fragments).  Weight gradients are FP32 reductions over the CTA's rows
// from shared memory, added to global FP32 gradients; Adam updates FP32 master
// weights and re-issues their BF16 copies.
#include <cuda_bf16.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <random>
#include <vector>

#include "../../include/glasma.h"
#include "ic.cuh"
#include "internal.h"

namespace glasma {

constexpr int MI = 36, MK1 = 48, MH = 128, MO = 16;
constexpr int MROWS = 64;  // rows per CTA (4 warps x 16)
constexpr int N_W1 = MH * MI, N_W2 = MH * MH, N_W3 = MO * MH;
constexpr int O_W1 = 0, O_B1 = O_W1 + N_W1, O_W2 = O_B1 + MH, O_B2 = O_W2 + N_W2, O_W3 = O_B2 + MH,
              O_B3 = O_W3 + N_W3, N_PARAMS = O_B3 + MO;

struct MlpDev {
    const __nv_bfloat16* w1;   // [128][48] (inputs padded to 48)
    const __nv_bfloat16* w2;   // [128][128]
    const __nv_bfloat16* w3;   // [16][128]
    const __nv_bfloat16* w2t;  // [128][128] transposed
    const __nv_bfloat16* w3t;  // [128][16]  transposed
    const float* p;            // FP32 master parameters (biases read from here)
    float x_inv, y_scale;
};

DEV uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}
DEV void mma_bf16(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
// B fragment of a weight stored [n][K] (K contiguous): column n of the K x N operand
DEV void bfrag(const __nv_bfloat16* w, int K, int nt, int kt, int g, int t, uint32_t& b0, uint32_t& b1) {
    const __nv_bfloat16* row = w + (size_t)(nt * 8 + g) * K + kt * 16 + 2 * t;
    b0 = *reinterpret_cast<const uint32_t*>(row);
    b1 = *reinterpret_cast<const uint32_t*>(row + 8);
}
// A fragments of the next layer from FP32 accumulator fragments c[2*kt], c[2*kt+1]
DEV void afrag_from_acc(const float c0[4], const float c1[4], uint32_t a[4]) {
    a[0] = pack_bf16(c0[0], c0[1]);
    a[1] = pack_bf16(c0[2], c0[3]);
    a[2] = pack_bf16(c1[0], c1[1]);
    a[3] = pack_bf16(c1[2], c1[3]);
}

struct MlpSmem {  // training: activations and gradients of the CTA's rows
    __nv_bfloat16 w1[MH * MK1], w2[MH * MH], w3[MO * MH], w2t[MH * MH], w3t[MH * MO];
    __nv_bfloat16 x[MROWS * MK1], h1[MROWS * MH], h2[MROWS * MH], d2[MROWS * MH], d1[MROWS * MH];
    float dy[MROWS * MO];
    float b1[MH], b2[MH], b3[MO];
};
struct MlpSmemInfer {  // inference: weights and one row tile (layers chain in registers)
    __nv_bfloat16 w1[MH * MK1], w2[MH * MH], w3[MO * MH];
    __nv_bfloat16 x[MROWS * MK1];
    float b1[MH], b2[MH], b3[MO];
};
template <bool TRAIN> struct MlpSmemOf { using type = MlpSmem; };
template <> struct MlpSmemOf<false> { using type = MlpSmemInfer; };

// Training (TRAIN): one 64-row tile per CTA, forward and backward.  Inference: a
// persistent grid, weights loaded once per CTA, row tiles strided over the grid.
template <bool TRAIN>
__global__ void __launch_bounds__(128) k_mlp(MlpDev m, const float* __restrict__ X, const float* __restrict__ Tg,
                                              int N, float* __restrict__ Y, float* __restrict__ grad,
                                              double* __restrict__ loss) {
    extern __shared__ __align__(16) unsigned char smraw[];
    using SM = typename MlpSmemOf<TRAIN>::type;
    SM& S = *reinterpret_cast<SM*>(smraw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
    // weights and biases into shared memory
    {
        const uint4* src[3] = {(const uint4*)m.w1, (const uint4*)m.w2, (const uint4*)m.w3};
        uint4* dst[3] = {(uint4*)S.w1, (uint4*)S.w2, (uint4*)S.w3};
        const int cnt[3] = {MH * MK1 / 8, MH * MH / 8, MO * MH / 8};
        for (int q = 0; q < 3; q++)
            for (int i = tid; i < cnt[q]; i += 128) dst[q][i] = src[q][i];
        if constexpr (TRAIN) {
            for (int i = tid; i < MH * MH / 8; i += 128) ((uint4*)S.w2t)[i] = ((const uint4*)m.w2t)[i];
            for (int i = tid; i < MH * MO / 8; i += 128) ((uint4*)S.w3t)[i] = ((const uint4*)m.w3t)[i];
        }
        for (int i = tid; i < MH; i += 128) { S.b1[i] = m.p[O_B1 + i]; S.b2[i] = m.p[O_B2 + i]; }
        if (tid < MO) S.b3[tid] = m.p[O_B3 + tid];
    }
    const int ntiles = (N + MROWS - 1) / MROWS;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        __syncthreads();  // weights in place; the previous tile's inputs consumed
        {
            // input rows (scaled, BF16, zero padded)
            const int r0 = tile * MROWS;
            for (int i = tid; i < MROWS * MK1; i += 128) {
                const int r = i / MK1, k = i % MK1;
                const float v = (r0 + r < N && k < MI) ? X[(size_t)(r0 + r) * MI + k] * m.x_inv : 0.0f;
                S.x[i] = __float2bfloat16_rn(v);
            }
        }
        __syncthreads();
        const int rw = warp * 16;  // this warp's rows within the CTA
        const int row0 = tile * MROWS + rw;
        // ---- layer 1
        float c1[16][4];
#pragma unroll
        for (int nt = 0; nt < 16; nt++) {
            const float b0 = S.b1[nt * 8 + 2 * t], b1v = S.b1[nt * 8 + 2 * t + 1];
            c1[nt][0] = b0; c1[nt][1] = b1v; c1[nt][2] = b0; c1[nt][3] = b1v;
        }
#pragma unroll
        for (int kt = 0; kt < MK1 / 16; kt++) {
            uint32_t a[4];
            const __nv_bfloat16* xr = S.x + (rw + g) * MK1 + kt * 16 + 2 * t;
            a[0] = *reinterpret_cast<const uint32_t*>(xr);
            a[1] = *reinterpret_cast<const uint32_t*>(xr + 8 * MK1);
            a[2] = *reinterpret_cast<const uint32_t*>(xr + 8);
            a[3] = *reinterpret_cast<const uint32_t*>(xr + 8 * MK1 + 8);
#pragma unroll
            for (int nt = 0; nt < 16; nt++) {
                uint32_t b0, b1;
                bfrag(S.w1, MK1, nt, kt, g, t, b0, b1);
                mma_bf16(c1[nt], a, b0, b1);
            }
        }
#pragma unroll
        for (int nt = 0; nt < 16; nt++)
#pragma unroll
            for (int q = 0; q < 4; q++) c1[nt][q] = tanhf(c1[nt][q]);
        if constexpr (TRAIN) {
#pragma unroll
            for (int nt = 0; nt < 16; nt++) {
                const int col = nt * 8 + 2 * t;
                *reinterpret_cast<uint32_t*>(S.h1 + (rw + g) * MH + col) = pack_bf16(c1[nt][0], c1[nt][1]);
                *reinterpret_cast<uint32_t*>(S.h1 + (rw + g + 8) * MH + col) = pack_bf16(c1[nt][2], c1[nt][3]);
            }
        }
        // ---- layer 2
        float c2[16][4];
#pragma unroll
        for (int nt = 0; nt < 16; nt++) {
            const float b0 = S.b2[nt * 8 + 2 * t], b1v = S.b2[nt * 8 + 2 * t + 1];
            c2[nt][0] = b0; c2[nt][1] = b1v; c2[nt][2] = b0; c2[nt][3] = b1v;
        }
#pragma unroll
        for (int kt = 0; kt < MH / 16; kt++) {
            uint32_t a[4];
            afrag_from_acc(c1[2 * kt], c1[2 * kt + 1], a);
#pragma unroll
            for (int nt = 0; nt < 16; nt++) {
                uint32_t b0, b1;
                bfrag(S.w2, MH, nt, kt, g, t, b0, b1);
                mma_bf16(c2[nt], a, b0, b1);
            }
        }
#pragma unroll
        for (int nt = 0; nt < 16; nt++)
#pragma unroll
            for (int q = 0; q < 4; q++) c2[nt][q] = tanhf(c2[nt][q]);
        if constexpr (TRAIN) {
#pragma unroll
            for (int nt = 0; nt < 16; nt++) {
                const int col = nt * 8 + 2 * t;
                *reinterpret_cast<uint32_t*>(S.h2 + (rw + g) * MH + col) = pack_bf16(c2[nt][0], c2[nt][1]);
                *reinterpret_cast<uint32_t*>(S.h2 + (rw + g + 8) * MH + col) = pack_bf16(c2[nt][2], c2[nt][3]);
            }
        }
        // ---- layer 3
        float c3[2][4];
#pragma unroll
        for (int nt = 0; nt < 2; nt++) {
            const float b0 = S.b3[nt * 8 + 2 * t], b1v = S.b3[nt * 8 + 2 * t + 1];
            c3[nt][0] = b0; c3[nt][1] = b1v; c3[nt][2] = b0; c3[nt][3] = b1v;
        }
#pragma unroll
        for (int kt = 0; kt < MH / 16; kt++) {
            uint32_t a[4];
            afrag_from_acc(c2[2 * kt], c2[2 * kt + 1], a);
#pragma unroll
            for (int nt = 0; nt < 2; nt++) {
                uint32_t b0, b1;
                bfrag(S.w3, MH, nt, kt, g, t, b0, b1);
                mma_bf16(c3[nt], a, b0, b1);
            }
        }
        const int ra = row0 + g, rb = row0 + g + 8;
        if constexpr (!TRAIN) {
            // outputs 0..7 (n-tile 0): delta = y * y_scale
            if (ra < N) {
                Y[(size_t)ra * 8 + 2 * t] = c3[0][0] * m.y_scale;
                Y[(size_t)ra * 8 + 2 * t + 1] = c3[0][1] * m.y_scale;
            }
            if (rb < N) {
                Y[(size_t)rb * 8 + 2 * t] = c3[0][2] * m.y_scale;
                Y[(size_t)rb * 8 + 2 * t + 1] = c3[0][3] * m.y_scale;
            }
        } else {
            // ---- loss and dY = 2 (y - target) / (N * 16); targets of outputs 8..15 are 0
            const float norm = 2.0f / ((float)N * MO);
            double lsum = 0.0;
            float dyf[2][4];
#pragma unroll
            for (int nt = 0; nt < 2; nt++)
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const int r = (q < 2) ? ra : rb;
                    const int col = nt * 8 + 2 * t + (q & 1);
                    float d = 0.0f;
                    if (r < N) {
                        const float tg = (nt == 0) ? Tg[(size_t)r * 8 + col] / m.y_scale : 0.0f;
                        const float e = c3[nt][q] - tg;
                        lsum += (double)e * e;
                        d = norm * e;
                    }
                    dyf[nt][q] = d;
                    S.dy[(rw + g + ((q < 2) ? 0 : 8)) * MO + col] = d;
                }
            // dH2 = (dY W3) * (1 - h2^2)
            {
                float d2[16][4];
                uint32_t a[4];
                afrag_from_acc(dyf[0], dyf[1], a);
#pragma unroll
                for (int nt = 0; nt < 16; nt++) {
                    d2[nt][0] = d2[nt][1] = d2[nt][2] = d2[nt][3] = 0.0f;
                    uint32_t b0, b1;
                    bfrag(S.w3t, MO, nt, 0, g, t, b0, b1);
                    mma_bf16(d2[nt], a, b0, b1);
#pragma unroll
                    for (int q = 0; q < 4; q++) d2[nt][q] *= 1.0f - c2[nt][q] * c2[nt][q];
                    const int col = nt * 8 + 2 * t;
                    *reinterpret_cast<uint32_t*>(S.d2 + (rw + g) * MH + col) = pack_bf16(d2[nt][0], d2[nt][1]);
                    *reinterpret_cast<uint32_t*>(S.d2 + (rw + g + 8) * MH + col) = pack_bf16(d2[nt][2], d2[nt][3]);
                }
            }
            __syncwarp();  // this warp's rows of S.d2 are complete
            // dH1 = (dH2 W2) * (1 - h1^2); dH2 operands and h1 come back from shared memory
            {
                float d1[16][4];
#pragma unroll
                for (int nt = 0; nt < 16; nt++) d1[nt][0] = d1[nt][1] = d1[nt][2] = d1[nt][3] = 0.0f;
#pragma unroll
                for (int kt = 0; kt < MH / 16; kt++) {
                    uint32_t a[4];
                    const __nv_bfloat16* dr = S.d2 + (rw + g) * MH + kt * 16 + 2 * t;
                    a[0] = *reinterpret_cast<const uint32_t*>(dr);
                    a[1] = *reinterpret_cast<const uint32_t*>(dr + 8 * MH);
                    a[2] = *reinterpret_cast<const uint32_t*>(dr + 8);
                    a[3] = *reinterpret_cast<const uint32_t*>(dr + 8 * MH + 8);
#pragma unroll
                    for (int nt = 0; nt < 16; nt++) {
                        uint32_t b0, b1;
                        bfrag(S.w2t, MH, nt, kt, g, t, b0, b1);
                        mma_bf16(d1[nt], a, b0, b1);
                    }
                }
#pragma unroll
                for (int nt = 0; nt < 16; nt++) {
                    const int col = nt * 8 + 2 * t;
                    const float h00 = __bfloat162float(S.h1[(rw + g) * MH + col]);
                    const float h01 = __bfloat162float(S.h1[(rw + g) * MH + col + 1]);
                    const float h10 = __bfloat162float(S.h1[(rw + g + 8) * MH + col]);
                    const float h11 = __bfloat162float(S.h1[(rw + g + 8) * MH + col + 1]);
                    d1[nt][0] *= 1.0f - h00 * h00;
                    d1[nt][1] *= 1.0f - h01 * h01;
                    d1[nt][2] *= 1.0f - h10 * h10;
                    d1[nt][3] *= 1.0f - h11 * h11;
                    *reinterpret_cast<uint32_t*>(S.d1 + (rw + g) * MH + col) = pack_bf16(d1[nt][0], d1[nt][1]);
                    *reinterpret_cast<uint32_t*>(S.d1 + (rw + g + 8) * MH + col) = pack_bf16(d1[nt][2], d1[nt][3]);
                }
            }
            // loss: warp sum -> one atomic per warp
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, o);
            if (lane == 0) atomicAdd(loss, lsum / ((double)N * MO));
            __syncthreads();
            // ---- weight gradients over this CTA's rows (FP32 accumulation from BF16 activations)
            {
                // W2 and b2: thread o = tid, columns in chunks of 32
                const int o = tid;
                float gb = 0.0f;
                for (int r = 0; r < MROWS; r++) gb += __bfloat162float(S.d2[r * MH + o]);
                atomicAdd(grad + O_B2 + o, gb);
                for (int c0 = 0; c0 < MH; c0 += 32) {
                    float acc[32];
#pragma unroll
                    for (int i = 0; i < 32; i++) acc[i] = 0.0f;
                    for (int r = 0; r < MROWS; r++) {
                        const float d = __bfloat162float(S.d2[r * MH + o]);
#pragma unroll
                        for (int i = 0; i < 32; i++) acc[i] = fmaf(d, __bfloat162float(S.h1[r * MH + c0 + i]), acc[i]);
                    }
#pragma unroll
                    for (int i = 0; i < 32; i++) atomicAdd(grad + O_W2 + o * MH + c0 + i, acc[i]);
                }
                // W1 and b1
                {
                    float acc[MI];
                    float gb1 = 0.0f;
#pragma unroll
                    for (int k = 0; k < MI; k++) acc[k] = 0.0f;
                    for (int r = 0; r < MROWS; r++) {
                        const float d = __bfloat162float(S.d1[r * MH + o]);
                        gb1 += d;
#pragma unroll
                        for (int k = 0; k < MI; k++) acc[k] = fmaf(d, __bfloat162float(S.x[r * MK1 + k]), acc[k]);
                    }
                    atomicAdd(grad + O_B1 + o, gb1);
#pragma unroll
                    for (int k = 0; k < MI; k++) atomicAdd(grad + O_W1 + o * MI + k, acc[k]);
                }
                // W3 and b3: o3 = tid & 15, columns (tid >> 4) * 16 .. + 16
                {
                    const int o3 = tid & 15, c0 = (tid >> 4) * 16;
                    float acc[16];
                    float gb3 = 0.0f;
#pragma unroll
                    for (int i = 0; i < 16; i++) acc[i] = 0.0f;
                    for (int r = 0; r < MROWS; r++) {
                        const float d = S.dy[r * MO + o3];
                        gb3 += d;
#pragma unroll
                        for (int i = 0; i < 16; i++) acc[i] = fmaf(d, __bfloat162float(S.h2[r * MH + c0 + i]), acc[i]);
                    }
                    if (c0 == 0) atomicAdd(grad + O_B3 + o3, gb3);
#pragma unroll
                    for (int i = 0; i < 16; i++) atomicAdd(grad + O_W3 + o3 * MH + c0 + i, acc[i]);
                }
            }
        }  // TRAIN
    }  // tiles
}

// Adam on the FP32 master parameters, then the BF16 copies (padded / transposed)
__global__ void k_adam(float* __restrict__ p, float* __restrict__ mo, float* __restrict__ ve,
                       const float* __restrict__ gr, float lr, float b1, float b2, float eps, float c1, float c2,
                       int update) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N_PARAMS) return;
    if (update) {
        const float g = gr[i];
        const float m = b1 * mo[i] + (1.0f - b1) * g;
        const float v = b2 * ve[i] + (1.0f - b2) * g * g;
        mo[i] = m;
        ve[i] = v;
        p[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
    }
}
__global__ void k_mlp_bf16(const float* __restrict__ p, __nv_bfloat16* w1, __nv_bfloat16* w2, __nv_bfloat16* w3,
                           __nv_bfloat16* w2t, __nv_bfloat16* w3t) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < MH * MK1) {
        const int o = i / MK1, k = i % MK1;
        w1[i] = __float2bfloat16_rn(k < MI ? p[O_W1 + o * MI + k] : 0.0f);
    }
    if (i < N_W2) {
        const int o = i / MH, c = i % MH;
        const __nv_bfloat16 v = __float2bfloat16_rn(p[O_W2 + i]);
        w2[i] = v;
        w2t[c * MH + o] = v;
    }
    if (i < N_W3) {
        const int o = i / MH, c = i % MH;
        const __nv_bfloat16 v = __float2bfloat16_rn(p[O_W3 + i]);
        w3[i] = v;
        w3t[c * MO + o] = v;
    }
}
// RMS of the inputs and targets (for the fixed scalings)
__global__ void k_sumsq(const float* __restrict__ a, size_t n, double* out) {
    double s = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double v = a[i];
        s += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

// ---------------------------------------------------------------- features, targets, warm starts
template <class T> DEV void put_features(const IcSeries<T>& q, float* f) {
    T s11 = 0, s22 = 0, s12 = 0, scc = 0;
#pragma unroll
    for (int a = 0; a < 8; a++) {
        f[a] = (float)q.a1.a[a];
        f[8 + a] = (float)q.a2.a[a];
        f[16 + a] = (float)q.c.a[a];
        f[24 + a] = (float)q.cubic.a[a];
        s11 += q.a1.a[a] * q.a1.a[a];
        s22 += q.a2.a[a] * q.a2.a[a];
        s12 += q.a1.a[a] * q.a2.a[a];
        scc += q.c.a[a] * q.c.a[a];
    }
    f[32] = (float)s11;
    f[33] = (float)s22;
    f[34] = (float)s12;
    f[35] = (float)scc;
}
// features of every link; with T (training data) also the targets, then in FP64
// throughout (the targets are differences of nearly equal offsets); without, in FP32
__global__ void k_ic_features(const double* __restrict__ V1, const double* __restrict__ V2, int n,
                              const double* __restrict__ U, float* __restrict__ X, float* __restrict__ T) {
    const size_t ns = (size_t)n * n;
    const size_t l = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (l >= 2 * ns) return;
    const size_t s = l >> 1;
    const int d = (int)(l & 1), x = (int)(s % n), y = (int)(s / n);
    const int xn = d == 0 ? (x == n - 1 ? 0 : x + 1) : x;
    const int yn = d == 1 ? (y == n - 1 ? 0 : y + 1) : y;
    const size_t s2 = xn + (size_t)n * yn;
    if (T) {
        const M3<double> U1 = mul_nd(ld18(V1 + 18 * s), ld18(V1 + 18 * s2));
        const M3<double> U2 = mul_nd(ld18(V2 + 18 * s), ld18(V2 + 18 * s2));
        const IcSeries<double> q = ic_series(U1, U2);
        put_features(q, X + 36 * l);
        // d^a = 2 Im Tr[t^a U (U1 U2)^dag] minus the series
        const Al<double> dl = im_tl(mul_nd(ld18(U + 36 * s + 18 * d), mul(U1, U2)));
        const Al<double> ds = series_offset(q);
#pragma unroll
        for (int a = 0; a < 8; a++) T[8 * l + a] = (float)(dl.a[a] - ds.a[a]);
    } else {
        const M3<float> U1 = mul_nd(to_f32(ld18(V1 + 18 * s)), to_f32(ld18(V1 + 18 * s2)));
        const M3<float> U2 = mul_nd(to_f32(ld18(V2 + 18 * s)), to_f32(ld18(V2 + 18 * s2)));
        put_features(ic_series(U1, U2), X + 36 * l);
    }
}

}  // namespace glasma

using namespace glasma;

struct glasma_mlp {
    float* p;     // FP32 masters
    float* m;     // Adam moments
    float* v;
    float* g;     // gradients
    __nv_bfloat16 *w1, *w2, *w3, *w2t, *w3t;
    double* dsc;  // scratch doubles (loss, sums)
    float x_scale = 1.0f, y_scale = 1.0f;
    cudaStream_t st;
    long long t = 0;  // Adam step
};

void glasma_set_error(const char* msg);
static glasma_status mfail(glasma_status s, const char* msg) {
    glasma_set_error(msg);
    return s;
}
#define MCK(call)                                                                  \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) return mfail(GLASMA_ERR_CUDA, cudaGetErrorString(e_)); \
    } while (0)

static size_t mlp_bytes() {
    return 4 * align256((size_t)N_PARAMS * 4) + align256(MH * MK1 * 2) + 2 * align256(MH * MH * 2) +
           2 * align256(MO * MH * 2) + 256 + 1024;
}

extern "C" int64_t glasma_mlp_workspace_bytes(void) { return (int64_t)mlp_bytes(); }

static cudaError_t refresh_bf16(glasma_mlp* M) {
    k_mlp_bf16<<<(MH * MH + 255) / 256, 256, 0, M->st>>>(M->p, M->w1, M->w2, M->w3, M->w2t, M->w3t);
    return cudaGetLastError();
}

extern "C" glasma_status glasma_mlp_create(void* ws, int64_t bytes, uint64_t seed, void* stream, glasma_mlp** out) {
    if (!ws || !out || ((uintptr_t)ws & 255) || bytes < (int64_t)mlp_bytes())
        return mfail(GLASMA_ERR_INVALID, "glasma_mlp_create: bad workspace");
    glasma_mlp* M = new (std::nothrow) glasma_mlp();
    if (!M) return mfail(GLASMA_ERR_INVALID, "host allocation failed");
    char* b = (char*)ws;
    auto take = [&](size_t n) { char* r = b; b += align256(n); return r; };
    M->p = (float*)take((size_t)N_PARAMS * 4);
    M->m = (float*)take((size_t)N_PARAMS * 4);
    M->v = (float*)take((size_t)N_PARAMS * 4);
    M->g = (float*)take((size_t)N_PARAMS * 4);
    M->w1 = (__nv_bfloat16*)take(MH * MK1 * 2);
    M->w2 = (__nv_bfloat16*)take(MH * MH * 2);
    M->w2t = (__nv_bfloat16*)take(MH * MH * 2);
    M->w3 = (__nv_bfloat16*)take(MO * MH * 2);
    M->w3t = (__nv_bfloat16*)take(MO * MH * 2);
    M->dsc = (double*)take(256);
    M->st = (cudaStream_t)stream;
    // Glorot-uniform weights, zero biases; the output layer starts small so that an
    // untrained network proposes the plain U1 U2 start
    std::mt19937_64 rng(seed);
    std::uniform_real_distribution<float> u(-1.0f, 1.0f);
    std::vector<float> h(N_PARAMS, 0.0f);
    const float a1 = sqrtf(6.0f / (MI + MH)), a2 = sqrtf(6.0f / (MH + MH)), a3 = 0.1f * sqrtf(6.0f / (MH + MO));
    for (int i = 0; i < N_W1; i++) h[O_W1 + i] = a1 * u(rng);
    for (int i = 0; i < N_W2; i++) h[O_W2 + i] = a2 * u(rng);
    for (int i = 0; i < N_W3; i++) h[O_W3 + i] = a3 * u(rng);
    MCK(cudaMemcpyAsync(M->p, h.data(), h.size() * 4, cudaMemcpyHostToDevice, M->st));
    MCK(cudaMemsetAsync(M->m, 0, (size_t)N_PARAMS * 4, M->st));
    MCK(cudaMemsetAsync(M->v, 0, (size_t)N_PARAMS * 4, M->st));
    MCK(refresh_bf16(M));
    MCK(cudaStreamSynchronize(M->st));
    *out = M;
    return GLASMA_OK;
}
extern "C" void glasma_mlp_destroy(glasma_mlp* M) { delete M; }

static MlpDev dev_view(const glasma_mlp* M) {
    MlpDev d;
    d.w1 = M->w1; d.w2 = M->w2; d.w3 = M->w3; d.w2t = M->w2t; d.w3t = M->w3t; d.p = M->p;
    d.x_inv = 1.0f / M->x_scale;
    d.y_scale = M->y_scale;
    return d;
}
template <bool TRAIN> static cudaError_t launch_mlp(const glasma_mlp* M, const float* X, const float* T, int64_t N,
                                                    float* Y, cudaStream_t st) {
    using SM = typename MlpSmemOf<TRAIN>::type;
    static bool attr = false;
    static int grid_cap = 0;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_mlp<TRAIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SM));
        if (e != cudaSuccess) return e;
        int dev = 0, sms = 0, per = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_mlp<TRAIN>, 128, sizeof(SM))) != cudaSuccess)
            return e;
        grid_cap = std::max(1, sms * per);
        attr = true;
    }
    if (N <= 0) return cudaSuccess;
    const long long tiles = (N + MROWS - 1) / MROWS;
    // training: one tile per CTA (the gradients are per-CTA sums); inference: a persistent grid
    const unsigned nb = (unsigned)(TRAIN ? tiles : std::min<long long>(tiles, grid_cap));
    k_mlp<TRAIN><<<nb, 128, sizeof(SM), st>>>(dev_view(M), X, T, (int)N, Y, M->g, M->dsc);
    return cudaGetLastError();
}

extern "C" glasma_status glasma_mlp_set_scales(glasma_mlp* M, float x_scale, float y_scale) {
    if (!M || !(x_scale > 0) || !(y_scale > 0)) return mfail(GLASMA_ERR_INVALID, "bad scales");
    M->x_scale = x_scale;
    M->y_scale = y_scale;
    return GLASMA_OK;
}

extern "C" glasma_status glasma_mlp_fit_scales(glasma_mlp* M, const float* X, const float* T, int64_t N) {
    if (!M || !X || !T || N <= 0) return mfail(GLASMA_ERR_INVALID, "bad arguments");
    MCK(cudaMemsetAsync(M->dsc, 0, 2 * sizeof(double), M->st));
    k_sumsq<<<304, 256, 0, M->st>>>(X, (size_t)N * 36, M->dsc);
    k_sumsq<<<304, 256, 0, M->st>>>(T, (size_t)N * 8, M->dsc + 1);
    double h[2];
    MCK(cudaMemcpyAsync(h, M->dsc, sizeof(h), cudaMemcpyDeviceToHost, M->st));
    MCK(cudaStreamSynchronize(M->st));
    M->x_scale = (float)fmax(sqrt(h[0] / ((double)N * 36)), 1e-30);
    M->y_scale = (float)fmax(sqrt(h[1] / ((double)N * 8)), 1e-30);
    return GLASMA_OK;
}

// loss and FP32 gradients of one batch (no update); grads_host may be NULL
extern "C" glasma_status glasma_mlp_loss_grad(glasma_mlp* M, const float* X, const float* T, int64_t N,
                                              double* loss, float* grads_host) {
    if (!M || !X || !T || N <= 0) return mfail(GLASMA_ERR_INVALID, "bad arguments");
    MCK(cudaMemsetAsync(M->g, 0, (size_t)N_PARAMS * 4, M->st));
    MCK(cudaMemsetAsync(M->dsc, 0, sizeof(double), M->st));
    MCK(launch_mlp<true>(M, X, T, N, nullptr, M->st));
    double l = 0;
    MCK(cudaMemcpyAsync(&l, M->dsc, sizeof(double), cudaMemcpyDeviceToHost, M->st));
    if (grads_host) MCK(cudaMemcpyAsync(grads_host, M->g, (size_t)N_PARAMS * 4, cudaMemcpyDeviceToHost, M->st));
    MCK(cudaStreamSynchronize(M->st));
    if (loss) *loss = l;
    return GLASMA_OK;
}

// mini-batch Adam over the N pairs for some epochs (batches in order, the caller shuffles)
extern "C" glasma_status glasma_mlp_train(glasma_mlp* M, const float* X, const float* T, int64_t N, int32_t epochs,
                                          int32_t batch, float lr, double* last_loss) {
    if (!M || !X || !T || N <= 0 || epochs < 1 || batch < MROWS) return mfail(GLASMA_ERR_INVALID, "bad arguments");
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int e = 0; e < epochs; e++) {
        MCK(cudaMemsetAsync(M->dsc, 0, sizeof(double), M->st));
        for (int64_t off = 0; off + batch <= N; off += batch) {
            MCK(cudaMemsetAsync(M->g, 0, (size_t)N_PARAMS * 4, M->st));
            MCK(launch_mlp<true>(M, X + off * 36, T + off * 8, batch, nullptr, M->st));
            M->t++;
            const float c1 = 1.0f - powf(b1, (float)M->t), c2 = 1.0f - powf(b2, (float)M->t);
            k_adam<<<(N_PARAMS + 255) / 256, 256, 0, M->st>>>(M->p, M->m, M->v, M->g, lr, b1, b2, eps, c1, c2, 1);
            MCK(refresh_bf16(M));
        }
    }
    double l = 0;
    MCK(cudaMemcpyAsync(&l, M->dsc, sizeof(double), cudaMemcpyDeviceToHost, M->st));
    MCK(cudaStreamSynchronize(M->st));
    if (last_loss) *last_loss = l * (double)batch / (double)((N / batch) * batch);
    return GLASMA_OK;
}

extern "C" glasma_status glasma_mlp_predict(glasma_mlp* M, const float* X, int64_t N, float* Y) {
    if (!M || !X || !Y || N < 0) return mfail(GLASMA_ERR_INVALID, "bad arguments");
    MCK(launch_mlp<false>(M, X, nullptr, N, Y, M->st));
    return GLASMA_OK;
}

extern "C" glasma_status glasma_mlp_get_params(glasma_mlp* M, float* host, float* scales) {
    if (!M || !host) return mfail(GLASMA_ERR_INVALID, "bad arguments");
    MCK(cudaMemcpyAsync(host, M->p, (size_t)N_PARAMS * 4, cudaMemcpyDeviceToHost, M->st));
    MCK(cudaStreamSynchronize(M->st));
    if (scales) { scales[0] = M->x_scale; scales[1] = M->y_scale; }
    return GLASMA_OK;
}
extern "C" glasma_status glasma_mlp_set_params(glasma_mlp* M, const float* host) {
    if (!M || !host) return mfail(GLASMA_ERR_INVALID, "bad arguments");
    MCK(cudaMemcpyAsync(M->p, host, (size_t)N_PARAMS * 4, cudaMemcpyHostToDevice, M->st));
    MCK(refresh_bf16(M));
    MCK(cudaStreamSynchronize(M->st));
    return GLASMA_OK;
}

// features and targets of every link of the last MV initial condition of a context
namespace glasma {
cudaError_t launch_ic_features(const ICScratch& s, int n, float* X, float* T, cudaStream_t st) {
    const size_t nl = 2 * (size_t)n * n;
    k_ic_features<<<(unsigned)((nl + 255) / 256), 256, 0, st>>>(s.V1, s.V2, n, s.U, X, T);
    return cudaGetLastError();
}
cudaError_t mlp_predict_dev(glasma_mlp* M, const float* X, int64_t N, float* Y, cudaStream_t st) {
    return launch_mlp<false>(M, X, nullptr, N, Y, st);
}
}  // namespace glasma
