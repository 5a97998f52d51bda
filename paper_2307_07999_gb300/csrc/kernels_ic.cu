// MV initial conditions on the device (Sec. 1 "Glasma" of arXiv:2307.07999):
// Philox charges -> Poisson (cuFFT) -> Wilson lines -> pure-gauge nucleus links
// -> Newton solve of the tau = 0+ links -> pi(0) -> state at step 1.
#include <cufft.h>
#include <vector>

#include "ic.cuh"
#include "internal.h"

namespace glasma {

size_t ic_scratch_bytes(int n, size_t fft_work_bytes) {
    const size_t ns = (size_t)n * n;
    return 2 * align256(ns * 18 * 8) + align256(ns * 8 * 16) + align256(ns * 36 * 8) + align256(ns * 8 * 8) +
           align256(2 * ns * 4) + align256(2 * ns * 8) + align256(fft_work_bytes) + align256(2 * ns * 36 * 4) +
           align256(2 * ns * 8 * 4) + 256;
}
ICScratch ic_layout(void* base, int n, size_t fft_work_bytes) {
    const size_t ns = (size_t)n * n;
    char* p = (char*)base;
    ICScratch s;
    s.V1 = (double*)p; p += align256(ns * 18 * 8);
    s.V2 = (double*)p; p += align256(ns * 18 * 8);
    s.fft = (double*)p; p += align256(ns * 8 * 16);
    s.U = (double*)p; p += align256(ns * 36 * 8);
    s.pi0 = (double*)p; p += align256(ns * 8 * 8);
    s.iters = (int*)p; p += align256(2 * ns * 4);
    s.res = (double*)p; p += align256(2 * ns * 8);
    s.fft_work = p;
    s.fft_work_bytes = fft_work_bytes;
    p += align256(fft_work_bytes);
    s.X = (float*)p; p += align256(2 * ns * 36 * 4);
    s.D = (float*)p;
    return s;
}

static bool make_plan(int n, cufftHandle* plan, size_t* work, const char** err) {
    if (cufftCreate(plan) != CUFFT_SUCCESS) { *err = "cufftCreate failed"; return false; }
    if (cufftSetAutoAllocation(*plan, 0) != CUFFT_SUCCESS) { *err = "cufftSetAutoAllocation failed"; cufftDestroy(*plan); return false; }
    int dims[2] = {n, n};
    if (cufftMakePlanMany(*plan, 2, dims, nullptr, 1, n * n, nullptr, 1, n * n, CUFFT_Z2Z, 8, work) != CUFFT_SUCCESS) {
        *err = "cufftMakePlanMany failed";
        cufftDestroy(*plan);
        return false;
    }
    return true;
}
size_t ic_fft_work_bytes(int n, const char** err) {
    cufftHandle plan;
    size_t work = 0;
    if (!make_plan(n, &plan, &work, err)) return (size_t)-1;
    cufftDestroy(plan);
    return work;
}

// rho^a for one (nucleus, sheet): buf[a][s] complex, imaginary part 0
__global__ void k_mv_charges(double2* __restrict__ buf, int n, int n_sheets, double sigma, uint2 key, int nucleus,
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
        buf[(size_t)(4 * k + 0) * ns + s] = make_double2(sigma * g0, 0.0);
        buf[(size_t)(4 * k + 1) * ns + s] = make_double2(sigma * g1, 0.0);
        buf[(size_t)(4 * k + 2) * ns + s] = make_double2(sigma * g2, 0.0);
        buf[(size_t)(4 * k + 3) * ns + s] = make_double2(sigma * g3, 0.0);
    }
}
// divide by (k~^2 + m^2) N^2 (the inverse transform is unnormalised); zero mode -> 0
__global__ void k_poisson_scale(double2* __restrict__ buf, int n, double m2) {
    const size_t ns = (size_t)n * n;
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= 8 * ns) return;
    const size_t s = i % ns;
    const int kx = (int)(s % n), ky = (int)(s / n);
    if (kx == 0 && ky == 0) { buf[i] = make_double2(0.0, 0.0); return; }
    const double sx = sinpi((double)kx / n), sy = sinpi((double)ky / n);
    const double f = 1.0 / ((4.0 * sx * sx + 4.0 * sy * sy + m2) * (double)ns);
    buf[i] = make_double2(buf[i].x * f, buf[i].y * f);
}
__global__ void k_set_identity(double* __restrict__ V, size_t count) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= count) return;
    st18(V + 18 * i, ident());
}
// V <- exp(-i Lambda) V
__global__ void k_wilson_accum(const double2* __restrict__ lam, double* __restrict__ V, int n) {
    const size_t ns = (size_t)n * n;
    const size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (s >= ns) return;
    Al<double> x;
#pragma unroll
    for (int a = 0; a < 8; a++) x.a[a] = -lam[(size_t)a * ns + s].x;
    st18(V + 18 * s, mul(expi(herm(x)), ld18(V + 18 * s)));
}
DEV M3<double> nucleus_link(const double* V, int n, int x, int y, int d) {
    const int xn = d == 0 ? (x == n - 1 ? 0 : x + 1) : x;
    const int yn = d == 1 ? (y == n - 1 ? 0 : y + 1) : y;
    return mul_nd(ld18(V + 18 * (x + (size_t)n * y)), ld18(V + 18 * (xn + (size_t)n * yn)));
}
// Newton solve per link.  Start: exp(i (d_s + delta).t) U1 U2 when a predicted
// correction delta is given (d_s the third-order series of ic.cuh), else U1 U2; on
// a stall, restart from U1 U2 (after a warm start) and then from 1.  The iteration
// count includes every attempt.
__global__ void k_links_solve(const double* __restrict__ V1, const double* __restrict__ V2, int n, double tol,
                              int max_iter, double* __restrict__ U, int* __restrict__ iters,
                              double* __restrict__ res, const float* __restrict__ delta) {
    const size_t ns = (size_t)n * n;
    const size_t l = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (l >= 2 * ns) return;
    const size_t s = l >> 1;
    const int d = (int)(l & 1);
    const int x = (int)(s % n), y = (int)(s / n);
    const M3<double> U1 = nucleus_link(V1, n, x, y, d), U2 = nucleus_link(V2, n, x, y, d);
    const M3<double> P = mul(U1, U2);
    M3<double> u = P;
    int spent = 0;
    double r;
    int it;
    if (delta) {
        Al<double> dl = series_offset(ic_series(U1, U2));
#pragma unroll
        for (int a = 0; a < 8; a++) dl.a[a] += (double)delta[8 * l + a];
        u = mul(expi(herm(dl)), P);
        it = newton_link(U1, U2, u, tol, max_iter, r);
        if (it < 0) {
            spent = max_iter;
            u = P;
            it = newton_link(U1, U2, u, tol, max_iter, r);
        }
    } else {
        it = newton_link(U1, U2, u, tol, max_iter, r);
    }
    if (it < 0) {
        spent += max_iter;
        u = ident();
        it = newton_link(U1, U2, u, tol, max_iter, r);
    }
    if (it >= 0) it += spent;
    st18(U + 36 * s + 18 * d, u);
    iters[l] = it;
    res[l] = r;
}
// pi(0) = -(i/4) sum_i {[(U-1)(U2^dag-U1^dag) - h.c.](x) + [(U^dag-1)(U2-U1) - h.c.](x-i)}
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
    cufftHandle plan;
    size_t work = 0;
    std::vector<int> it_h;
    if (!make_plan(n, &plan, &work, err)) return -2;
    if (work > s.fft_work_bytes) { *err = "cuFFT work area larger than reserved"; cufftDestroy(plan); return -6; }
    if (cufftSetWorkArea(plan, s.fft_work) != CUFFT_SUCCESS || cufftSetStream(plan, st) != CUFFT_SUCCESS) {
        *err = "cufftSetWorkArea/SetStream failed";
        cufftDestroy(plan);
        return -2;
    }
    for (int A = 0; A < 2; A++) {
        double* V = A == 0 ? s.V1 : s.V2;
        k_set_identity<<<nb, 256, 0, st>>>(V, ns);
        for (int sh = 0; sh < n_sheets; sh++) {
            double2* fb = (double2*)s.fft;
            k_mv_charges<<<nb, 256, 0, st>>>(fb, n, n_sheets, sigma, key, A, sh);
            if (cufftExecZ2Z(plan, (cufftDoubleComplex*)fb, (cufftDoubleComplex*)fb, CUFFT_FORWARD) != CUFFT_SUCCESS) {
                *err = "cufftExecZ2Z forward failed";
                goto fail;
            }
            k_poisson_scale<<<(int)((8 * ns + 255) / 256), 256, 0, st>>>(fb, n, m_ir_a * m_ir_a);
            if (cufftExecZ2Z(plan, (cufftDoubleComplex*)fb, (cufftDoubleComplex*)fb, CUFFT_INVERSE) != CUFFT_SUCCESS) {
                *err = "cufftExecZ2Z inverse failed";
                goto fail;
            }
            k_wilson_accum<<<nb, 256, 0, st>>>(fb, V, n);
        }
    }
    if (mlp) {
        IC_CHECK(launch_ic_features(s, n, s.X, nullptr, st));
        IC_CHECK(mlp_predict_dev(mlp, s.X, (int64_t)(2 * ns), s.D, st));
    }
    k_links_solve<<<(int)((2 * ns + 63) / 64), 64, 0, st>>>(s.V1, s.V2, n, tol, max_iter, s.U, s.iters, s.res,
                                                            mlp ? s.D : nullptr);
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
    cufftDestroy(plan);
    return 0;
fail:
    cufftDestroy(plan);
    return -2;
}

}  // namespace glasma
