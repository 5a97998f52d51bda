// Lattice-correlator estimators of the momentum broadening (Sec. 2, "Lattice
// correlators", Eqs. 4 and 5 of arXiv:2307.07999), advanced with every field step.
//
//   static quarks (m -> infinity):  I_i(x) += dtau * E_i(x, tau_n)  at every site,
//                                   <dp_i^2> = < (1/2) sum_a (I_i^a)^2 >_x
//   lightlike jets along +x:        the path from x0 sits in cell x0 + k(m) after m steps,
//                                   J_i(x0) += dtau * W F_i W^dag, W <- W U_x(c) on leaving c,
//                                   F = (E_x, E_y - B_z, E_z + B_y),
//                                   <dp_i^2> = < (1/2) sum_a (J_i^a)^2 >_x0
// with the site-centred fields of the particle push (time-centred E, clover B_z from the
// plaquettes the field step stored, covariant differences of phi).  One thread per site;
// accumulators and Wilson lines in planes of n*n (component-major), in the precision of
// the fields; the six sums of each step reduce in FP64.
#include "internal.h"
#include "particles.cuh"

namespace glasma {

template <class T> struct CorrArgs {
    const T* fo;   // fields at step n
    const T* fn;   // fields at step n+1
    int n;
    T te;          // tau_n (expanding) or 1
    T dtau;
    T* I;          // [24][ns] static integrals
    T* J;          // [24][ns] lightlike integrals
    T* W;          // [18][ns] path Wilson lines (row-major entries, re/im)
    int k_now, k_next;
    double* acc;   // this step's row: {static x, y, z, lightlike x, y, z}
};

// Blocks of 128 threads; in FP32 at least 4 per SM (128 registers, 224 B of spills): the
// step waits on its gathers and its 66 accumulator planes, so resident warps decide it (field
// step + estimators on 1024^2: 757 us against 866 at 3 blocks and 1149 at the kernel's own
// 180 registers, 2 blocks).  FP64 keeps its registers.
template <class T> struct CorrMinb { static constexpr int v = 1; };
template <> struct CorrMinb<float> { static constexpr int v = 4; };
template <class T> __global__ void __launch_bounds__(128, CorrMinb<T>::v) k_corr_step(CorrArgs<T> A) {
    const int n = A.n;
    const size_t ns = (size_t)n * n;
    const size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    double part[6] = {0, 0, 0, 0, 0, 0};
    if (s < ns) {
        const int x = (int)(s % n), y = (int)(s / n);
        const GlobalSrc<T, false, true> F{A.fo, A.fn, n, ns};  // fo holds its plaquettes (one-event step)
        {  // static: the site's own fields
            Al<T> E[3];
            site_E(F.view(x, y), A.te, E);
#pragma unroll
            for (int i = 0; i < 3; i++) {
                double q = 0;
#pragma unroll
                for (int a = 0; a < 8; a++) {
                    T* p = A.I + (size_t)(8 * i + a) * ns + s;
                    const T v = *p + A.dtau * E[i].a[a];
                    *p = v;
                    q += (double)v * v;
                }
                part[i] = 0.5 * q;
            }
        }
        {  // lightlike: the path from (x, y) is in cell (x + k_now, y)
            const int cx = (int)(((long long)x + A.k_now) % n);
            const auto C = F.view(cx, y);
            Al<T> E[3], B[3];
            site_fields(C, A.te, E, B);
            Al<T> Fl[3];
#pragma unroll
            for (int a = 0; a < 8; a++) {
                Fl[0].a[a] = E[0].a[a];
                Fl[1].a[a] = E[1].a[a] - B[2].a[a];
                Fl[2].a[a] = E[2].a[a] + B[1].a[a];
            }
            M3<T> W;
#pragma unroll
            for (int e = 0; e < 9; e++)
                W.m[e / 3][e % 3] = mk(A.W[(size_t)(2 * e) * ns + s], A.W[(size_t)(2 * e + 1) * ns + s]);
#pragma unroll
            for (int i = 0; i < 3; i++) {
                const Al<T> t = conj_alg(W, Fl[i]);  // W F W^dag
                double q = 0;
#pragma unroll
                for (int a = 0; a < 8; a++) {
                    T* p = A.J + (size_t)(8 * i + a) * ns + s;
                    const T v = *p + A.dtau * t.a[a];
                    *p = v;
                    q += (double)v * v;
                }
                part[3 + i] = 0.5 * q;
            }
            if (A.k_next > A.k_now) {
                const M3<T> Wn = mul(W, C.link(0, 0, 0));
#pragma unroll
                for (int e = 0; e < 9; e++) {
                    A.W[(size_t)(2 * e) * ns + s] = Wn.m[e / 3][e % 3].r;
                    A.W[(size_t)(2 * e + 1) * ns + s] = Wn.m[e / 3][e % 3].i;
                }
            }
        }
    }
    // warp -> block -> one FP64 atomic per block and sum
#pragma unroll
    for (int i = 0; i < 6; i++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part[i] += __shfl_down_sync(0xffffffffu, part[i], o);
    __shared__ double red[6][4];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0)
#pragma unroll
        for (int i = 0; i < 6; i++) red[i][w] = part[i];
    __syncthreads();
    if (threadIdx.x < 6) {
        double t = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += red[threadIdx.x][k];
        atomicAdd(A.acc + threadIdx.x, t);
    }
}

template <class T> __global__ void k_corr_reset(T* I, T* J, T* W, size_t ns) {
    const size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (s >= ns) return;
    for (int k = 0; k < 24; k++) {
        I[(size_t)k * ns + s] = T(0);
        J[(size_t)k * ns + s] = T(0);
    }
    for (int k = 0; k < 18; k++) W[(size_t)k * ns + s] = (k == 0 || k == 8 || k == 16) ? T(1) : T(0);
}

size_t corr_state_bytes(int prec, int n) { return (size_t)66 * n * n * (prec ? 4 : 8); }

cudaError_t launch_corr_reset(int prec, void* state, int n, cudaStream_t st) {
    const size_t ns = (size_t)n * n;
    const unsigned nb = (unsigned)((ns + 127) / 128);
    if (prec) {
        float* b = (float*)state;
        k_corr_reset<float><<<nb, 128, 0, st>>>(b, b + 24 * ns, b + 48 * ns, ns);
    } else {
        double* b = (double*)state;
        k_corr_reset<double><<<nb, 128, 0, st>>>(b, b + 24 * ns, b + 48 * ns, ns);
    }
    return cudaGetLastError();
}

template <class T>
static cudaError_t corr_impl(const void* fo, const void* fn, int n, double te, double dtau, void* state, int k_now,
                             int k_next, double* acc, cudaStream_t st) {
    const size_t ns = (size_t)n * n;
    CorrArgs<T> A;
    A.fo = (const T*)fo;
    A.fn = (const T*)fn;
    A.n = n;
    A.te = (T)te;
    A.dtau = (T)dtau;
    A.I = (T*)state;
    A.J = A.I + 24 * ns;
    A.W = A.I + 48 * ns;
    A.k_now = k_now;
    A.k_next = k_next;
    A.acc = acc;
    k_corr_step<T><<<(unsigned)((ns + 127) / 128), 128, 0, st>>>(A);
    return cudaGetLastError();
}
cudaError_t launch_corr_step(int prec, const void* fo, const void* fn, int n, double te, double dtau, void* state,
                             int k_now, int k_next, double* acc, cudaStream_t st) {
    return prec ? corr_impl<float>(fo, fn, n, te, dtau, state, k_now, k_next, acc, st)
                : corr_impl<double>(fo, fn, n, te, dtau, state, k_now, k_next, acc, st);
}

}  // namespace glasma
