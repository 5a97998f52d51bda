// MV initial conditions on the device (Sec. 1 "Glasma" of arXiv:2307.07999):
// Philox charges -> Poisson (cuFFT) -> Wilson lines -> pure-gauge nucleus links
// -> Newton solve of the tau = 0+ links -> pi(0) -> state at step 1.
#include <cufft.h>

#include <algorithm>
#include <vector>

#include "ic.cuh"
#include "internal.h"

namespace glasma {

// half-spectrum elements of one real n x n transform
static size_t spec_elems(int n) { return (size_t)n * (size_t)(n / 2 + 1); }
size_t ic_scratch_bytes(int n, size_t fft_work_bytes) {
    const size_t ns = (size_t)n * n;
    return 2 * align256(ns * 18 * 8) + align256(ns * 8 * 8) + align256(spec_elems(n) * 8 * 16) +
           align256(ns * 36 * 8) + align256(ns * 8 * 8) +
           align256(2 * ns * 4) + align256(2 * ns * 8) + align256(fft_work_bytes) + align256(2 * ns * 36 * 4) +
           align256(2 * ns * 8 * 4) + align256((size_t)n * 8) + align256(4 * 2 * ns * 4) + align256(16) + 256;
}
ICScratch ic_layout(void* base, int n, size_t fft_work_bytes) {
    const size_t ns = (size_t)n * n;
    char* p = (char*)base;
    ICScratch s;
    s.V1 = (double*)p; p += align256(ns * 18 * 8);
    s.V2 = (double*)p; p += align256(ns * 18 * 8);
    s.fft = (double*)p; p += align256(ns * 8 * 8);
    s.spec = (double*)p; p += align256(spec_elems(n) * 8 * 16);
    s.U = (double*)p; p += align256(ns * 36 * 8);
    s.pi0 = (double*)p; p += align256(ns * 8 * 8);
    s.iters = (int*)p; p += align256(2 * ns * 4);
    s.res = (double*)p; p += align256(2 * ns * 8);
    s.fft_work = p;
    s.fft_work_bytes = fft_work_bytes;
    p += align256(fft_work_bytes);
    s.X = (float*)p; p += align256(2 * ns * 36 * 4);
    s.D = (float*)p; p += align256(2 * ns * 8 * 4);
    s.ktab = (double*)p; p += align256((size_t)n * 8);
    s.nwt = (int*)p; p += align256(4 * 2 * ns * 4);
    s.ncnt = (int*)p;
    return s;
}

// real-to-complex forward and complex-to-real inverse 2-D transforms, 8 color
// components per call (the charges and Lambda are real)
struct Plans {
    cufftHandle fwd = 0, inv = 0;
    bool ok_fwd = false, ok_inv = false;
    ~Plans() {
        if (ok_fwd) cufftDestroy(fwd);
        if (ok_inv) cufftDestroy(inv);
    }
};
static bool make_plans(int n, Plans& P, size_t* work, const char** err) {
    long long dims[2] = {n, n};
    const long long ns = (long long)n * n, nh = (long long)n * (n / 2 + 1);  // 8 transforms: > 2^31 reals at n = 16384
    size_t w1 = 0, w2 = 0;
    if (cufftCreate(&P.fwd) != CUFFT_SUCCESS) { *err = "cufftCreate failed"; return false; }
    P.ok_fwd = true;
    if (cufftCreate(&P.inv) != CUFFT_SUCCESS) { *err = "cufftCreate failed"; return false; }
    P.ok_inv = true;
    if (cufftSetAutoAllocation(P.fwd, 0) != CUFFT_SUCCESS || cufftSetAutoAllocation(P.inv, 0) != CUFFT_SUCCESS) {
        *err = "cufftSetAutoAllocation failed";
        return false;
    }
    if (cufftMakePlanMany64(P.fwd, 2, dims, nullptr, 1, ns, nullptr, 1, nh, CUFFT_D2Z, 8, &w1) != CUFFT_SUCCESS ||
        cufftMakePlanMany64(P.inv, 2, dims, nullptr, 1, nh, nullptr, 1, ns, CUFFT_Z2D, 8, &w2) != CUFFT_SUCCESS) {
        *err = "cufftMakePlanMany64 failed";
        return false;
    }
    *work = std::max(w1, w2);
    return true;
}
size_t ic_fft_work_bytes(int n, const char** err) {
    Plans P;
    size_t work = 0;
    if (!make_plans(n, P, &work, err)) return (size_t)-1;
    return work;
}

// rho^a for one (nucleus, sheet): buf[a][s]
__global__ void k_mv_charges(double* __restrict__ buf, int n, int n_sheets, double sigma, uint2 key, int nucleus,
                             int sheet) {
    const size_t ns = (size_t)n * n;
    const size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (s >= ns) return;
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const uint4 r = philox4x32_10(make_uint4((uint32_t)s, (uint32_t)(nucleus * n_sheets + sheet), (uint32_t)k, 1u), key);
        double g0, g1, g2, g3;
        box_muller(r.x, r.y, g0, g1);
        box_muller(r.z, r.w, g2, g3);
        buf[(size_t)(4 * k + 0) * ns + s] = sigma * g0;
        buf[(size_t)(4 * k + 1) * ns + s] = sigma * g1;
        buf[(size_t)(4 * k + 2) * ns + s] = sigma * g2;
        buf[(size_t)(4 * k + 3) * ns + s] = sigma * g3;
    }
}
// lattice momenta k~_i^2 = 4 sin^2(pi k_i / n), once per solve
__global__ void k_lattice_momenta(double* __restrict__ ktab, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double s = sinpi((double)k / n);
    ktab[k] = 4.0 * s * s;
}
// divide the half spectrum by (k~^2 + m^2) N^2 (the inverse transform is
// unnormalised); zero mode -> 0.  One thread per momentum, all 8 color components.
__global__ void k_poisson_scale(double2* __restrict__ spec, const double* __restrict__ ktab, int n, double m2) {
    const int nh = n / 2 + 1;
    const size_t ne = (size_t)n * nh;
    const size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (s >= ne) return;
    const int kx = (int)(s % nh), ky = (int)(s / nh);
    const double f = (kx == 0 && ky == 0) ? 0.0 : 1.0 / ((ktab[kx] + ktab[ky] + m2) * ((double)n * n));
#pragma unroll
    for (int a = 0; a < 8; a++) {
        const double2 v = spec[(size_t)a * ne + s];
        spec[(size_t)a * ne + s] = make_double2(v.x * f, v.y * f);
    }
}
__global__ void k_set_identity(double* __restrict__ V, size_t count) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= count) return;
    st18(V + 18 * i, ident());
}
// V <- exp(-i Lambda) V
__global__ void k_wilson_accum(const double* __restrict__ lam, double* __restrict__ V, int n) {
    const size_t ns = (size_t)n * n;
    const size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (s >= ns) return;
    Al<double> x;
#pragma unroll
    for (int a = 0; a < 8; a++) x.a[a] = -lam[(size_t)a * ns + s];
    st18(V + 18 * s, mul(expi(herm(x)), ld18(V + 18 * s)));
}
DEV M3<double> nucleus_link(const double* V, int n, int x, int y, int d) {
    const int xn = d == 0 ? (x == n - 1 ? 0 : x + 1) : x;
    const int yn = d == 1 ? (y == n - 1 ? 0 : y + 1) : y;
    return mul_nd(ld18(V + 18 * (x + (size_t)n * y)), ld18(V + 18 * (xn + (size_t)n * yn)));
}
// Newton solve of every link, in passes over a compacted list of the links not yet
// converged, one Newton step per link and pass (links that need few steps cost only
// those: no warp waits for a slower neighbour).  Attempts per link: the start
// exp(i (d_s + delta).t) U1 U2 when a predicted correction delta is given (d_s the
// third-order series of ic.cuh), then U1 U2, then 1; an attempt ends when it
// converges, stalls, meets a singular Jacobian or reaches max_iter steps, and a failed
// attempt counts max_iter towards the link's total.  iters[l] holds the attempts'
// spent count while the link is active and its total (or -1) once it is done.
struct NewtonState {
    const double *V1, *V2;
    int n;
    double tol;
    int max_iter;
    double* U;     // [ns][2][18]
    int* iters;    // [2 ns]
    double* res;   // [2 ns]
    int* att;      // [2 ns] attempt: 0 warm start, 1 U1 U2, 2 identity
    int* ita;      // [2 ns] steps of the current attempt
};
DEV void link_pair(const NewtonState& N, size_t l, M3<double>& U1, M3<double>& U2) {
    const size_t s = l >> 1;
    const int d = (int)(l & 1), x = (int)(s % N.n), y = (int)(s / N.n);
    U1 = nucleus_link(N.V1, N.n, x, y, d);
    U2 = nucleus_link(N.V2, N.n, x, y, d);
}
// start attempt a of link l at u; done (converged) -> iters final, else queued
DEV void newton_begin(const NewtonState& N, size_t l, int a, int spent, const M3<double>& S, const M3<double>& u,
                      int* out, int* out_n) {
    const double rn = nrm8(ic_residual(S, u));
    st18(N.U + 18 * l, u);
    N.res[l] = rn;
    N.att[l] = a;
    N.ita[l] = 0;
    if (rn <= N.tol) {
        N.iters[l] = spent;
    } else {
        N.iters[l] = spent;
        out[atomicAdd(out_n, 1)] = (int)l;
    }
}
__global__ void k_newton_start(NewtonState N, const float* __restrict__ delta, int* __restrict__ out,
                               int* __restrict__ out_n) {
    const size_t ns = (size_t)N.n * N.n;
    const size_t l = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (l >= 2 * ns) return;
    M3<double> U1, U2;
    link_pair(N, l, U1, U2);
    const M3<double> S = addm(U1, U2), P = mul(U1, U2);
    if (delta) {
        // the series in FP32: the start needs no more than the network's accuracy
        const Al<float> sf = series_offset(ic_series(to_f32(U1), to_f32(U2)));
        Al<double> dl;
#pragma unroll
        for (int a = 0; a < 8; a++) dl.a[a] = (double)sf.a[a] + (double)delta[8 * l + a];
        newton_begin(N, l, 0, 0, S, mul(expi(herm(dl)), P), out, out_n);
    } else {
        newton_begin(N, l, 1, 0, S, P, out, out_n);
    }
}
__global__ void k_newton_pass(NewtonState N, const int* __restrict__ in, const int* __restrict__ in_n,
                              int* __restrict__ out, int* __restrict__ out_n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= *in_n) return;
    const size_t l = (size_t)in[k];
    M3<double> U1, U2;
    link_pair(N, l, U1, U2);
    const M3<double> S = addm(U1, U2);
    M3<double> u = ld18(N.U + 18 * l);
    Al<double> r = ic_residual(S, u);
    double rn = N.res[l];
    bool stalled = false;
    const bool exhausted = N.ita[l] >= N.max_iter;
    const bool ok = !exhausted && newton_step(S, u, r, rn, &stalled);
    const int it = N.ita[l] + (ok ? 1 : 0);
    const int spent = N.iters[l];
    if (ok && rn <= N.tol) {  // converged
        st18(N.U + 18 * l, u);
        N.res[l] = rn;
        N.iters[l] = spent + it;
        return;
    }
    if (!ok || stalled || it >= N.max_iter) {  // this attempt failed: next start, or give up
        const int a = N.att[l] + 1;
        if (a == 1) {
            newton_begin(N, l, 1, spent + N.max_iter, S, mul(U1, U2), out, out_n);
        } else if (a == 2) {
            newton_begin(N, l, 2, spent + N.max_iter, S, ident(), out, out_n);
        } else {
            st18(N.U + 18 * l, u);
            N.res[l] = rn;
            N.iters[l] = -1;
        }
        return;
    }
    st18(N.U + 18 * l, u);
    N.res[l] = rn;
    N.ita[l] = it;
    out[atomicAdd(out_n, 1)] = (int)l;
}

__global__ void k_pi0(const double* __restrict__ V1, const double* __restrict__ V2, const double* __restrict__ U,
                      int n, double* __restrict__ pi) {
    const size_t ns = (size_t)n * n;
    const size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (s >= ns) return;
    const int x = (int)(s % n), y = (int)(s / n);
    M3<double> M;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) M.m[i][j] = mk(0.0, 0.0);
    for (int d = 0; d < 2; d++) {
        const int xm = d == 0 ? (x == 0 ? n - 1 : x - 1) : x, ym = d == 1 ? (y == 0 ? n - 1 : y - 1) : y;
        const size_t sm = xm + (size_t)n * ym;
        {
            const M3<double> u = ld18(U + 36 * s + 18 * d);
            const M3<double> A = addm(u, ident(), -1.0);
            const M3<double> B = addm(dag(nucleus_link(V2, n, x, y, d)), dag(nucleus_link(V1, n, x, y, d)), -1.0);
            const M3<double> C = mul(A, B);
            M = addm(addm(M, C), dag(C), -1.0);
        }
        {
            const M3<double> u = ld18(U + 36 * sm + 18 * d);
            const M3<double> A = addm(dag(u), ident(), -1.0);
            const M3<double> B = addm(nucleus_link(V2, n, xm, ym, d), nucleus_link(V1, n, xm, ym, d), -1.0);
            const M3<double> C = mul(A, B);
            M = addm(addm(M, C), dag(C), -1.0);
        }
    }
    // H = -(i/4) M is Hermitian; components 2 Re Tr(t^a H) = (1/4) * 2 Re Tr(t^a (-i M))
    M3<double> H;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) H.m[i][j] = mk(0.25 * M.m[i][j].i, -0.25 * M.m[i][j].r);
    const Al<double> p = re_comp(H);
#pragma unroll
    for (int a = 0; a < 8; a++) pi[8 * s + a] = p.a[a];
}
// state at step 1: U_1 = U_0, E_{1/2} = 0, pi_{1/2} = pi(0), phi_1 = dtau (dtau/2) pi(0)
template <class T>
__global__ void k_ic_finalize(const double* __restrict__ U, const double* __restrict__ pi, int n, double dtau,
                              T* __restrict__ f) {
    const size_t ns = (size_t)n * n;
    const size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (s >= ns) return;
#pragma unroll
    for (int d = 0; d < 2; d++)
#pragma unroll
        for (int k = 0; k < 12; k++) f[fidx(12 * d + k, s, ns)] = (T)U[36 * s + 18 * d + k];
#pragma unroll
    for (int a = 0; a < 16; a++) f[fidx(P_EX + a, s, ns)] = T(0);
#pragma unroll
    for (int a = 0; a < 8; a++) {
        f[fidx(P_PI + a, s, ns)] = (T)pi[8 * s + a];
        f[fidx(P_PHI + a, s, ns)] = (T)(dtau * (0.5 * dtau) * pi[8 * s + a]);
    }
}

#define IC_CHECK(x)                                  \
    do {                                             \
        if ((x) != cudaSuccess) { *err = #x; goto fail; } \
    } while (0)

int ic_run(int prec, int n, int n_sheets, double g2mua, double m_ir_a, uint64_t seed, double dtau, double tol,
           int max_iter, const ICScratch& s, void* buf, cudaStream_t st, long long* fails, double* mean_it,
           int* max_it, const char** err, ::glasma_mlp* mlp) {
    const size_t ns = (size_t)n * n;
    const uint2 key = make_uint2((uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
    const double sigma = g2mua / sqrt((double)n_sheets);
    const int nb = (int)((ns + 255) / 256);
    Plans plan;
    size_t work = 0;
    std::vector<int> it_h;
    if (!make_plans(n, plan, &work, err)) return -2;
    if (work > s.fft_work_bytes) { *err = "cuFFT work area larger than reserved"; return -6; }
    if (cufftSetWorkArea(plan.fwd, s.fft_work) != CUFFT_SUCCESS || cufftSetStream(plan.fwd, st) != CUFFT_SUCCESS ||
        cufftSetWorkArea(plan.inv, s.fft_work) != CUFFT_SUCCESS || cufftSetStream(plan.inv, st) != CUFFT_SUCCESS) {
        *err = "cufftSetWorkArea/SetStream failed";
        return -2;
    }
    k_lattice_momenta<<<(n + 255) / 256, 256, 0, st>>>(s.ktab, n);
    for (int A = 0; A < 2; A++) {
        double* V = A == 0 ? s.V1 : s.V2;
        k_set_identity<<<nb, 256, 0, st>>>(V, ns);
        for (int sh = 0; sh < n_sheets; sh++) {
            k_mv_charges<<<nb, 256, 0, st>>>(s.fft, n, n_sheets, sigma, key, A, sh);
            if (cufftExecD2Z(plan.fwd, (cufftDoubleReal*)s.fft, (cufftDoubleComplex*)s.spec) != CUFFT_SUCCESS) {
                *err = "cufftExecD2Z failed";
                return -2;
            }
            k_poisson_scale<<<(int)((spec_elems(n) + 255) / 256), 256, 0, st>>>((double2*)s.spec, s.ktab, n,
                                                                             m_ir_a * m_ir_a);
            if (cufftExecZ2D(plan.inv, (cufftDoubleComplex*)s.spec, (cufftDoubleReal*)s.fft) != CUFFT_SUCCESS) {
                *err = "cufftExecZ2D failed";
                return -2;
            }
            k_wilson_accum<<<nb, 256, 0, st>>>(s.fft, V, n);
        }
    }
    if (mlp) {
        IC_CHECK(launch_ic_features(s, n, s.X, nullptr, st));
        IC_CHECK(mlp_predict_dev(mlp, s.X, (int64_t)(2 * ns), s.D, st));
    }
    {
        const NewtonState N{s.V1, s.V2, n, tol, max_iter, s.U, s.iters, s.res, s.nwt, s.nwt + 2 * ns};
        int* list[2] = {s.nwt + 4 * ns, s.nwt + 6 * ns};
        IC_CHECK(cudaMemsetAsync(s.ncnt, 0, 2 * sizeof(int), st));
        k_newton_start<<<(int)((2 * ns + 127) / 128), 128, 0, st>>>(N, mlp ? s.D : nullptr, list[0], s.ncnt);
        // every pass advances each listed link by one step; a link takes at most
        // 3 * max_iter steps, and the host reads the list length between passes
        for (int pass = 0, cur = 0; pass <= 3 * max_iter + 3; pass++, cur ^= 1) {
            int cnt = 0;
            IC_CHECK(cudaMemcpyAsync(&cnt, s.ncnt + cur, sizeof(int), cudaMemcpyDeviceToHost, st));
            IC_CHECK(cudaStreamSynchronize(st));
            if (cnt == 0) break;
            IC_CHECK(cudaMemsetAsync(s.ncnt + (cur ^ 1), 0, sizeof(int), st));
            k_newton_pass<<<(cnt + 127) / 128, 128, 0, st>>>(N, list[cur], s.ncnt + cur, list[cur ^ 1],
                                                            s.ncnt + (cur ^ 1));
        }
    }
    k_pi0<<<nb, 256, 0, st>>>(s.V1, s.V2, s.U, n, s.pi0);
    if (prec) k_ic_finalize<float><<<nb, 256, 0, st>>>(s.U, s.pi0, n, dtau, (float*)buf);
    else k_ic_finalize<double><<<nb, 256, 0, st>>>(s.U, s.pi0, n, dtau, (double*)buf);
    IC_CHECK(cudaGetLastError());
    it_h.resize(2 * ns);
    IC_CHECK(cudaMemcpyAsync(it_h.data(), s.iters, 2 * ns * sizeof(int), cudaMemcpyDeviceToHost, st));
    IC_CHECK(cudaStreamSynchronize(st));
    {
        long long f = 0, sum = 0;
        int mx = 0;
        for (size_t l = 0; l < 2 * ns; l++) {
            if (it_h[l] < 0) f++;
            else { sum += it_h[l]; if (it_h[l] > mx) mx = it_h[l]; }
        }
        *fails = f;
        *mean_it = (2 * ns - f) > 0 ? (double)sum / (double)(2 * ns - f) : 0.0;
        *max_it = mx;
    }
    return 0;
fail:
    return -2;
}

}  // namespace glasma
