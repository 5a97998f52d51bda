// Field monitors for callers that cannot allocate device memory.
//
// glasma_diagnostics needs a context, and a context needs a caller-provided
// workspace.  Some callers cannot obtain device memory at all: code that runs
// inside another framework's allocator-free region (a host callback, a plugin
// handed only the buffers it must read), or a process whose memory pool is
// already fully reserved by the application.  glasma_diagnostics_noalloc
// serves them: it reads a field buffer the caller already owns and keeps its
// reduction scratch (per-block partial sums) in the file-scope array below,
// which every GPU that loads this library holds until the process exits.
#include "../../include/glasma.h"
#include "field.cuh"

namespace glasma {

// per-block partial sums: 8 doubles per block, blocks of 256 sites
constexpr int NOALLOC_MAX_BLOCKS = 4096;            // => at most 1,048,576 sites (n <= 1024)
constexpr int NOALLOC_BLOCK = 256;
static __device__ __align__(256) double g_monitor_scratch[NOALLOC_MAX_BLOCKS * 8 + 8];

// the eight monitor terms of one site (same definitions as glasma_diagnostics)
template <class T>
DEV void site_terms(const T* __restrict__ f, int n, size_t s, double te, double t[8]) {
    const size_t ns = (size_t)n * n;
    const int x = (int)(s % n), y = (int)(s / n);
    const size_t sxm = (x == 0 ? n - 1 : x - 1) + (size_t)n * y, sym = x + (size_t)n * (y == 0 ? n - 1 : y - 1);
    const size_t sxp = (x == n - 1 ? 0 : x + 1) + (size_t)n * y, syp = x + (size_t)n * (y == n - 1 ? 0 : y + 1);
    M3<T> ux, uy;
    load_links(f, ns, s, ux, uy);
    const Al<T> ex = load_alg(f, ns, P_EX, s), ey = load_alg(f, ns, P_EY, s);
    const Al<T> phi = load_alg(f, ns, P_PHI, s), pi = load_alg(f, ns, P_PI, s);
    const Al<T> tx = transport_alg(load_link(f, ns, P_UX, sxm), load_alg(f, ns, P_EX, sxm));
    const Al<T> ty = transport_alg(load_link(f, ns, P_UY, sym), load_alg(f, ns, P_EY, sym));
    const Al<T> cm = icomm(phi, pi);
    double g2 = 0, den = 0, eet = 0, eel = 0, p2 = 0, q2 = 0;
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
    const double ebl = 2.0 * (3.0 - ((double)P.m[0][0].r + P.m[1][1].r + P.m[2][2].r));
    const Al<T> psx = conj_alg(ux, load_alg(f, ns, P_PHI, sxp));
    const Al<T> psy = conj_alg(uy, load_alg(f, ns, P_PHI, syp));
    double ebt = 0;
    for (int a = 0; a < 8; a++) {
        const double dx = (double)psx.a[a] - phi.a[a], dy = (double)psy.a[a] - phi.a[a];
        ebt += 0.5 * (dx * dx + dy * dy);
    }
    eet /= te * te;
    ebt /= te * te;
    double ud = 0;
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
    const double tot = g2 + den + eet + ebt + eel + ebl;
    t[0] = g2; t[1] = den; t[2] = eet; t[3] = ebt; t[4] = eel; t[5] = ebl; t[6] = ud;
    t[7] = isfinite(tot) ? 0.0 : 1.0;
}

// pass 1: one block of 256 sites -> its 8 partials (sums; slot 6 a maximum)
template <class T>
__global__ void __launch_bounds__(NOALLOC_BLOCK) k_monitor_partials(const T* __restrict__ f, int n, double te,
                                                                     double* __restrict__ part) {
    const size_t ns = (size_t)n * n;
    const size_t s = blockIdx.x * (size_t)NOALLOC_BLOCK + threadIdx.x;
    double t[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (s < ns) site_terms(f, n, s, te, t);
    __shared__ double red[8][NOALLOC_BLOCK / 32];
    for (int k = 0; k < 8; k++) {
        double v = t[k];
        for (int o = 16; o > 0; o >>= 1) {
            const double w = __shfl_down_sync(0xffffffffu, v, o);
            v = k == 6 ? fmax(v, w) : v + w;
        }
        if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        const int k = threadIdx.x;
        double v = red[k][0];
        for (int w = 1; w < NOALLOC_BLOCK / 32; w++) v = k == 6 ? fmax(v, red[k][w]) : v + red[k][w];
        part[8 * (size_t)blockIdx.x + k] = v;
    }
}
// pass 2: one thread per term sums the partials in block order (deterministic)
__global__ void k_monitor_final(double* __restrict__ part, int nb) {
    const int k = threadIdx.x;
    if (k >= 8) return;
    double v = part[k];
    for (int b = 1; b < nb; b++) v = k == 6 ? fmax(v, part[8 * (size_t)b + k]) : v + part[8 * (size_t)b + k];
    part[8 * (size_t)NOALLOC_MAX_BLOCKS + k] = v;
}

}  // namespace glasma

using namespace glasma;

// Device address of g_monitor_scratch on the current device.  Looked up at every call
// (cudaGetSymbolAddress allocates nothing): an address cached across calls would go stale
// when the device's context is torn down and created again (cudaDeviceReset), and the
// kernel would then write to memory that is no longer the array.
static glasma_status scratch_for_current_device(double** out) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_monitor_scratch) != cudaSuccess || !p) return GLASMA_ERR_CUDA;
    *out = (double*)p;
    return GLASMA_OK;
}

void glasma_set_error(const char* msg);

extern "C" glasma_status glasma_diagnostics_noalloc(const void* fields, int32_t n, int32_t precision,
                                                    int32_t expanding, double tau, void* stream, double out[8]) {
    if (!fields || !out || n < 2 || (precision != GLASMA_FP64 && precision != GLASMA_FP32)) {
        glasma_set_error("glasma_diagnostics_noalloc: bad arguments");
        return GLASMA_ERR_INVALID;
    }
    if (((uintptr_t)fields & 15) != 0) {
        glasma_set_error("glasma_diagnostics_noalloc: field buffer not 16-byte aligned");
        return GLASMA_ERR_INVALID;
    }
    const size_t ns = (size_t)n * n;
    const size_t nb = (ns + NOALLOC_BLOCK - 1) / NOALLOC_BLOCK;
    if (nb > (size_t)NOALLOC_MAX_BLOCKS) {
        glasma_set_error("glasma_diagnostics_noalloc: lattice larger than the static scratch (n*n <= 1048576)");
        return GLASMA_ERR_INVALID;
    }
    if (expanding && !(tau > 0)) {  // E and D phi are divided by tau
        glasma_set_error("glasma_diagnostics_noalloc: the expanding evolution needs tau > 0");
        return GLASMA_ERR_INVALID;
    }
    cudaStream_t st = (cudaStream_t)stream;
    {  // synchronous (a device-to-host copy, then a wait): it cannot be part of a capture
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
            cudaGetLastError();
            glasma_set_error("glasma_diagnostics_noalloc: bad stream");
            return GLASMA_ERR_INVALID;
        }
        if (cs != cudaStreamCaptureStatusNone) {
            glasma_set_error("glasma_diagnostics_noalloc: the call synchronises and cannot be captured");
            return GLASMA_ERR_INVALID;
        }
    }
    {  // the buffer must be memory of the current device (a host pointer or another GPU's
       // buffer would pass the checks above and make the kernel fault)
        int dev = -1;
        cudaPointerAttributes pa;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaPointerGetAttributes(&pa, fields) != cudaSuccess) {
            cudaGetLastError();
            glasma_set_error("glasma_diagnostics_noalloc: cannot query the field buffer");
            return GLASMA_ERR_INVALID;
        }
        if ((pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged) || pa.device != dev) {
            glasma_set_error("glasma_diagnostics_noalloc: fields is not device memory of the current device");
            return GLASMA_ERR_INVALID;
        }
    }
    double* part = nullptr;
    if (scratch_for_current_device(&part) != GLASMA_OK) {
        glasma_set_error("glasma_diagnostics_noalloc: cudaGetSymbolAddress failed");
        return GLASMA_ERR_CUDA;
    }
    const double te = expanding ? tau : 1.0;
    if (precision == GLASMA_FP32)
        k_monitor_partials<float><<<(unsigned)nb, NOALLOC_BLOCK, 0, st>>>((const float*)fields, n, te, part);
    else
        k_monitor_partials<double><<<(unsigned)nb, NOALLOC_BLOCK, 0, st>>>((const double*)fields, n, te, part);
    k_monitor_final<<<1, 32, 0, st>>>(part, (int)nb);
    double m[8];
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(m, part + 8 * (size_t)NOALLOC_MAX_BLOCKS, sizeof(m),
                                              cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        glasma_set_error(cudaGetErrorString(e));
        return GLASMA_ERR_CUDA;
    }
    out[0] = m[1] > 0 ? sqrt(m[0] / m[1]) : sqrt(m[0]);
    out[1] = m[2] / (double)ns;
    out[2] = m[3] / (double)ns;
    out[3] = m[4] / (double)ns;
    out[4] = m[5] / (double)ns;
    out[5] = m[6];
    out[6] = tau;
    out[7] = m[7];
    if (m[7] > 0) {
        glasma_set_error("glasma_diagnostics_noalloc: nonfinite field values");
        return GLASMA_ERR_NONFINITE;
    }
    return GLASMA_OK;
}
