// C ABI of the library (declared in include/glasma.h).  Host orchestration
// only: every step of the method runs in the kernels of the kernels_*.cu files.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "../../include/glasma.h"
#include "internal.h"

using namespace glasma;

static thread_local char g_err[512] = "";
static glasma_status fail(glasma_status s, const char* fmt, const char* a = "") {
    snprintf(g_err, sizeof(g_err), fmt, a);
    return s;
}
static glasma_status cuda_fail(cudaError_t e, const char* where) {
    snprintf(g_err, sizeof(g_err), "%s: %s", where, cudaGetErrorString(e));
    return GLASMA_ERR_CUDA;
}
#define CK(call)                                                     \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);          \
    } while (0)

extern "C" const char* glasma_last_error(void) { return g_err; }
void glasma_set_error(const char* msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }

static const double HBARC = 0.1973269804;  // GeV fm

// device workspace bump allocator
struct Arena {
    char* base;
    size_t size, off;
    void* take(size_t b) {
        off = align256(off);
        if (off + b > size) return nullptr;
        void* p = base + off;
        off += b;
        return p;
    }
};

struct glasma_corr;
struct glasma_ctx {
    glasma_corr* corr = nullptr;  // attached lattice-correlator estimators (advance with every field step)
    glasma_params p;
    int n;
    size_t ns;
    int prec;
    size_t rs;
    void* buf[2];
    int cur;
    int step;
    int n_steps;
    double a_fm, a_gev, dtau;
    cudaStream_t st;
    double* mon;
    void* ic_base;
    size_t fft_work;
    long long ic_fails;
    double ic_mean;
    int ic_max;
};

static glasma_status check_params(const glasma_params* p) {
    if (!p) return fail(GLASMA_ERR_INVALID, "null params");
    if (p->n < 2 || p->n > 16384) return fail(GLASMA_ERR_INVALID, "n must be in [2, 16384]");
    if (!(p->L_fm > 0) || !(p->dtau_over_a > 0) || p->dtau_over_a > 1.0)
        return fail(GLASMA_ERR_INVALID, "L_fm > 0 and 0 < dtau_over_a <= 1 required");
    if (p->precision != GLASMA_FP64 && p->precision != GLASMA_FP32) return fail(GLASMA_ERR_INVALID, "bad precision");
    if (p->n_sheets < 1 || p->n_sheets > 4096) return fail(GLASMA_ERR_INVALID, "n_sheets out of range");
    if (!(p->tau_end_fm > 0)) return fail(GLASMA_ERR_INVALID, "tau_end_fm must be > 0");
    return GLASMA_OK;
}
static size_t field_buf_bytes(const glasma_params* p) {
    const size_t rs = p->precision == GLASMA_FP32 ? 4 : 8;
    return align256((size_t)N_FIELD_PLANES * (size_t)p->n * p->n * rs);
}

extern "C" int64_t glasma_workspace_bytes(const glasma_params* p) {
    glasma_status s = check_params(p);
    if (s != GLASMA_OK) return s;
    const char* err = "";
    const size_t work = ic_fft_work_bytes(p->n, &err);
    if (work == (size_t)-1) return fail(GLASMA_ERR_CUDA, "%s", err);
    return (int64_t)(2 * field_buf_bytes(p) + 256 + ic_scratch_bytes(p->n, work) + 1024);
}

extern "C" glasma_status glasma_create(const glasma_params* p, void* ws, int64_t ws_bytes, void* stream,
                                       glasma_ctx** out) {
    glasma_status s = check_params(p);
    if (s != GLASMA_OK) return s;
    if (!ws || !out || ((uintptr_t)ws & 255)) return fail(GLASMA_ERR_INVALID, "workspace must be non-null, 256-byte aligned");
    const int64_t need = glasma_workspace_bytes(p);
    if (need < 0) return (glasma_status)need;
    if (ws_bytes < need) return fail(GLASMA_ERR_NOSPACE, "workspace too small");
    glasma_ctx* g = new (std::nothrow) glasma_ctx();
    if (!g) return fail(GLASMA_ERR_INVALID, "host allocation failed");
    g->p = *p;
    g->n = p->n;
    g->ns = (size_t)p->n * p->n;
    g->prec = p->precision;
    g->rs = g->prec ? 4 : 8;
    Arena A{(char*)ws, (size_t)ws_bytes, 0};
    g->buf[0] = A.take(field_buf_bytes(p));
    g->buf[1] = A.take(field_buf_bytes(p));
    g->mon = (double*)A.take(256);
    const char* err = "";
    g->fft_work = ic_fft_work_bytes(p->n, &err);
    g->ic_base = A.take(ic_scratch_bytes(p->n, g->fft_work));
    if (!g->buf[0] || !g->buf[1] || !g->mon || !g->ic_base) { delete g; return fail(GLASMA_ERR_NOSPACE, "workspace too small"); }
    g->cur = 0;
    g->step = -1;
    g->a_fm = p->L_fm / p->n;
    g->a_gev = g->a_fm / HBARC;
    g->dtau = p->dtau_over_a;
    g->n_steps = (int)ceil(p->tau_end_fm / (g->dtau * g->a_fm) - 1e-9);
    g->st = (cudaStream_t)stream;
    *out = g;
    return GLASMA_OK;
}

static void corr_detach(glasma_ctx* g);
extern "C" void glasma_destroy(glasma_ctx* g) {
    if (!g) return;
    corr_detach(g);
    delete g;
}

static glasma_status init_impl(glasma_ctx* g, glasma_mlp* mlp) {
    if (!g) return fail(GLASMA_ERR_INVALID, "null context");
    if (!g->p.expanding) return fail(GLASMA_ERR_INVALID, "MV initial conditions need the expanding evolution");
    const ICScratch sc = ic_layout(g->ic_base, g->n, g->fft_work);
    const char* err = "";
    const int tol_it = g->p.newton_max_iter > 0 ? g->p.newton_max_iter : 100;
    const double tol = g->p.newton_tol > 0 ? g->p.newton_tol : 1e-12;
    int rc = ic_run(g->prec, g->n, g->p.n_sheets, g->p.g2mu_GeV * g->a_gev, g->p.m_ir_GeV * g->a_gev, g->p.seed,
                    g->dtau, tol, tol_it, sc, g->buf[0], g->st, &g->ic_fails, &g->ic_mean, &g->ic_max, &err, mlp);
    if (rc == -6) return fail(GLASMA_ERR_NOSPACE, "%s", err);
    if (rc != 0) return fail(GLASMA_ERR_CUDA, "%s", err);
    g->cur = 0;
    g->step = 1;
    return g->ic_fails ? fail(GLASMA_ERR_NOCONV, "some tau=0+ links did not converge") : GLASMA_OK;
}

extern "C" glasma_status glasma_init(glasma_ctx* g) { return init_impl(g, nullptr); }

extern "C" glasma_status glasma_init_warm(glasma_ctx* g, glasma_mlp* mlp) {
    if (!mlp) return fail(GLASMA_ERR_INVALID, "null network");
    return init_impl(g, mlp);
}

extern "C" glasma_status glasma_ic_dataset(glasma_ctx* g, float* X, float* T) {
    if (!g || !X || !T) return fail(GLASMA_ERR_INVALID, "null argument");
    if (g->step < 0) return fail(GLASMA_ERR_INVALID, "no initial condition to read");
    const ICScratch sc = ic_layout(g->ic_base, g->n, g->fft_work);
    CK(launch_ic_features(sc, g->n, X, T, g->st));
    CK(cudaStreamSynchronize(g->st));
    return GLASMA_OK;
}

extern "C" glasma_status glasma_ic_stats(const glasma_ctx* g, int64_t* failures, double* mean_iter, int32_t* max_iter) {
    if (!g) return fail(GLASMA_ERR_INVALID, "null context");
    if (failures) *failures = g->ic_fails;
    if (mean_iter) *mean_iter = g->ic_mean;
    if (max_iter) *max_iter = g->ic_max;
    return GLASMA_OK;
}

// canonical host arrays pass through the IC scratch region as a staging area
extern "C" glasma_status glasma_init_from_host(glasma_ctx* g, const double* U, const double* E, const double* phi,
                                               const double* pi, int32_t step) {
    if (!g || !U || !E || !phi || !pi) return fail(GLASMA_ERR_INVALID, "null argument");
    if (step < 1 && g->p.expanding) return fail(GLASMA_ERR_INVALID, "expanding evolution needs step >= 1");
    const size_t ns = g->ns;
    double* d = (double*)g->ic_base;  // needs 36+16+8+8 = 68 doubles per site (< IC scratch)
    double *dU = d, *dE = d + 36 * ns, *dphi = dE + 16 * ns, *dpi = dphi + 8 * ns;
    CK(cudaMemcpyAsync(dU, U, 36 * ns * 8, cudaMemcpyHostToDevice, g->st));
    CK(cudaMemcpyAsync(dE, E, 16 * ns * 8, cudaMemcpyHostToDevice, g->st));
    CK(cudaMemcpyAsync(dphi, phi, 8 * ns * 8, cudaMemcpyHostToDevice, g->st));
    CK(cudaMemcpyAsync(dpi, pi, 8 * ns * 8, cudaMemcpyHostToDevice, g->st));
    CK(launch_state_from_canonical(g->prec, dU, dE, dphi, dpi, g->buf[0], g->n, g->st));
    CK(cudaStreamSynchronize(g->st));
    g->cur = 0;
    g->step = step;
    return GLASMA_OK;
}

extern "C" glasma_status glasma_get_state(glasma_ctx* g, double* U, double* E, double* phi, double* pi,
                                          int32_t* step) {
    if (!g) return fail(GLASMA_ERR_INVALID, "null context");
    if (g->step < 0) return fail(GLASMA_ERR_INVALID, "state not initialised");
    const size_t ns = g->ns;
    double* d = (double*)g->ic_base;
    double *dU = d, *dE = d + 36 * ns, *dphi = dE + 16 * ns, *dpi = dphi + 8 * ns;
    CK(launch_state_to_canonical(g->prec, g->buf[g->cur], U ? dU : nullptr, E ? dE : nullptr, phi ? dphi : nullptr,
                                 pi ? dpi : nullptr, g->n, g->st));
    if (U) CK(cudaMemcpyAsync(U, dU, 36 * ns * 8, cudaMemcpyDeviceToHost, g->st));
    if (E) CK(cudaMemcpyAsync(E, dE, 16 * ns * 8, cudaMemcpyDeviceToHost, g->st));
    if (phi) CK(cudaMemcpyAsync(phi, dphi, 8 * ns * 8, cudaMemcpyDeviceToHost, g->st));
    if (pi) CK(cudaMemcpyAsync(pi, dpi, 8 * ns * 8, cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    if (step) *step = g->step;
    return GLASMA_OK;
}

static glasma_status corr_after_step(glasma_ctx* g, const void* fo, const void* fn);
static glasma_status one_field_step(glasma_ctx* g) {
    const int reunit = reunit_code(g->p.reunit_every, g->step);
    const StepHost a = step_coeffs(g->buf[g->cur], g->buf[g->cur ^ 1], g->n, g->step, g->dtau, g->p.expanding, reunit);
    CK(launch_field_step(g->prec, a, g->st));
    if (g->corr) {
        glasma_status s = corr_after_step(g, g->buf[g->cur], g->buf[g->cur ^ 1]);
        if (s != GLASMA_OK) return s;
    }
    g->cur ^= 1;
    g->step++;
    return GLASMA_OK;
}

extern "C" glasma_status glasma_step(glasma_ctx* g, int32_t n_steps) {
    if (!g || n_steps < 0) return fail(GLASMA_ERR_INVALID, "bad arguments");
    if (g->step < 0) return fail(GLASMA_ERR_INVALID, "state not initialised");
    if (g->p.expanding && g->step < 1) return fail(GLASMA_ERR_INVALID, "expanding step needs tau > 0");
    for (int k = 0; k < n_steps; k++) {
        glasma_status s = one_field_step(g);
        if (s != GLASMA_OK) return s;
    }
    return GLASMA_OK;
}

extern "C" glasma_status glasma_diagnostics(glasma_ctx* g, double out[8]) {
    if (!g || !out) return fail(GLASMA_ERR_INVALID, "bad arguments");
    if (g->step < 0) return fail(GLASMA_ERR_INVALID, "state not initialised");
    const double tau = g->step * g->dtau;
    CK(launch_monitors(g->prec, g->buf[g->cur], g->n, g->p.expanding ? tau : 1.0, g->mon, g->st));
    double m[8];
    CK(cudaMemcpyAsync(m, g->mon, sizeof(m), cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    const double ns = (double)g->ns;
    out[0] = m[1] > 0 ? sqrt(m[0] / m[1]) : sqrt(m[0]);
    out[1] = m[2] / ns;
    out[2] = m[3] / ns;
    out[3] = m[4] / ns;
    out[4] = m[5] / ns;
    out[5] = m[6];
    out[6] = tau;
    out[7] = m[7];
    return m[7] > 0 ? fail(GLASMA_ERR_NONFINITE, "nonfinite field values") : GLASMA_OK;
}

// ------------------------------------------------------------------ particles
struct cpic_ctx {
    glasma_ctx* g;
    cpic_params p;
    int np;
    int n_form;
    PartHost P[2];
    int pcur;
    double* acc;     // [n_steps + 1][4]
    int acc_rows;
    int* sort_ws;
    double* stage;   // 17 * np doubles
    double* cas;     // 2 doubles
    double mass;
    int since_sort;
    int first_step;  // first pushed step: max(n_form, field step at particle initialisation)
};

static glasma_status check_cpic(const cpic_params* p) {
    if (!p) return fail(GLASMA_ERR_INVALID, "null params");
    if (p->n_particles < 0) return fail(GLASMA_ERR_INVALID, "n_particles < 0");
    if (p->mass_GeV < 0 || p->tau_form_fm < 0 || p->p_min_GeV < 0 || p->p_max_GeV < p->p_min_GeV)
        return fail(GLASMA_ERR_INVALID, "bad mass, tau_form or momentum range");
    if (p->init_kind != 0 && p->init_kind != 1) return fail(GLASMA_ERR_INVALID, "bad init_kind");
    if (p->integrator != 0 && p->integrator != 1) return fail(GLASMA_ERR_INVALID, "bad integrator");
    if (p->substeps < 0 || p->substeps > 64) return fail(GLASMA_ERR_INVALID, "substeps must be in [0, 64]");
    if (p->interp != 0 && p->interp != 1) return fail(GLASMA_ERR_INVALID, "bad interp");
    return GLASMA_OK;
}
static int total_steps(const glasma_params* gp) {
    const double a_fm = gp->L_fm / gp->n;
    return (int)ceil(gp->tau_end_fm / (gp->dtau_over_a * a_fm) - 1e-9);
}

extern "C" int64_t cpic_workspace_bytes(const glasma_params* gp, const cpic_params* p) {
    glasma_status s = check_params(gp);
    if (s != GLASMA_OK) return s;
    s = check_cpic(p);
    if (s != GLASMA_OK) return s;
    const int np = p->n_particles;
    const size_t ncell = (size_t)gp->n * gp->n;
    return (int64_t)(2 * part_bytes(np, gp->precision) + align256(((size_t)total_steps(gp) + 2) * 4 * 8) +
                     align256(sort_scratch_ints((int)ncell) * 4) + align256((size_t)17 * np * 8) + 256 + 2048);
}

extern "C" glasma_status cpic_create(glasma_ctx* g, const cpic_params* p, void* ws, int64_t ws_bytes, cpic_ctx** out) {
    if (!g || !out) return fail(GLASMA_ERR_INVALID, "null argument");
    glasma_status s = check_cpic(p);
    if (s != GLASMA_OK) return s;
    if (!ws || ((uintptr_t)ws & 255)) return fail(GLASMA_ERR_INVALID, "workspace must be non-null, 256-byte aligned");
    if (ws_bytes < cpic_workspace_bytes(&g->p, p)) return fail(GLASMA_ERR_NOSPACE, "workspace too small");
    cpic_ctx* c = new (std::nothrow) cpic_ctx();
    if (!c) return fail(GLASMA_ERR_INVALID, "host allocation failed");
    c->g = g;
    c->p = *p;
    c->np = p->n_particles;
    Arena A{(char*)ws, (size_t)ws_bytes, 0};
    const size_t pb = part_bytes(c->np, g->prec);
    c->P[0] = part_layout(A.take(pb), c->np, g->prec);
    c->P[1] = part_layout(A.take(pb), c->np, g->prec);
    c->acc_rows = g->n_steps + 2;
    c->acc = (double*)A.take((size_t)c->acc_rows * 4 * 8);
    c->sort_ws = (int*)A.take(sort_scratch_ints((int)g->ns) * 4);
    c->stage = (double*)A.take((size_t)17 * c->np * 8 + 8);
    c->cas = (double*)A.take(256);
    c->pcur = 0;
    c->n_form = (int)lround(p->tau_form_fm / (g->dtau * g->a_fm));
    if (c->n_form < 1) c->n_form = 1;
    c->mass = p->mass_GeV * g->a_gev;
    c->since_sort = 0;
    c->first_step = c->n_form;
    *out = c;
    return GLASMA_OK;
}
extern "C" void cpic_destroy(cpic_ctx* c) { delete c; }

extern "C" glasma_status cpic_init(cpic_ctx* c) {
    if (!c) return fail(GLASMA_ERR_INVALID, "null context");
    glasma_ctx* g = c->g;
    CK(launch_part_init(g->prec, c->P[0], c->np, g->n, c->p.init_kind, c->p.p_min_GeV * g->a_gev,
                        c->p.p_max_GeV * g->a_gev, c->p.q2, c->p.q3, c->p.seed, c->mass, g->st));
    CK(cudaMemsetAsync(c->acc, 0, (size_t)c->acc_rows * 4 * 8, g->st));
    c->pcur = 0;
    c->first_step = g->step > c->n_form ? g->step : c->n_form;
    return GLASMA_OK;
}

extern "C" glasma_status cpic_init_from_host(cpic_ctx* c, const double* x, const double* y, const double* eta,
                                             const double* px, const double* py, const double* peta, const double* Q,
                                             const double* p0) {
    if (!c || !x || !y || !eta || !px || !py || !peta || !Q || !p0) return fail(GLASMA_ERR_INVALID, "null argument");
    glasma_ctx* g = c->g;
    const size_t np = c->np;
    std::vector<double> h(17 * np);
    memcpy(h.data(), x, np * 8);
    memcpy(h.data() + np, y, np * 8);
    memcpy(h.data() + 2 * np, eta, np * 8);
    memcpy(h.data() + 3 * np, px, np * 8);
    memcpy(h.data() + 4 * np, py, np * 8);
    memcpy(h.data() + 5 * np, peta, np * 8);
    for (size_t j = 0; j < np; j++) {
        for (int a = 0; a < 8; a++) h[(6 + a) * np + j] = Q[8 * j + a];
        for (int k = 0; k < 3; k++) h[(14 + k) * np + j] = p0[3 * j + k];
    }
    CK(cudaMemcpyAsync(c->stage, h.data(), 17 * np * 8, cudaMemcpyHostToDevice, g->st));
    CK(launch_part_from_canonical(g->prec, c->P[0], c->np, g->n, c->stage, g->st));
    CK(cudaMemsetAsync(c->acc, 0, (size_t)c->acc_rows * 4 * 8, g->st));
    CK(cudaStreamSynchronize(g->st));
    c->pcur = 0;
    c->first_step = g->step > c->n_form ? g->step : c->n_form;
    return GLASMA_OK;
}

extern "C" glasma_status cpic_get_particles(cpic_ctx* c, double* x, double* y, double* eta, double* px, double* py,
                                            double* peta, double* Q) {
    if (!c) return fail(GLASMA_ERR_INVALID, "null context");
    glasma_ctx* g = c->g;
    const size_t np = c->np;
    CK(launch_part_to_canonical(g->prec, c->P[c->pcur], c->np, g->n, c->stage, g->st));
    std::vector<double> h(14 * np);
    CK(cudaMemcpyAsync(h.data(), c->stage, 14 * np * 8, cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    double* outs[6] = {x, y, eta, px, py, peta};
    for (int k = 0; k < 6; k++)
        if (outs[k]) memcpy(outs[k], h.data() + k * np, np * 8);
    if (Q)
        for (size_t j = 0; j < np; j++)
            for (int a = 0; a < 8; a++) Q[8 * j + a] = h[(6 + a) * np + j];
    return GLASMA_OK;
}

// the push of ensemble c from step n (fields fo) to n+1 (fields in the current buffer)
static PushHost push_host(const cpic_ctx* c, int n, const void* fo) {
    const glasma_ctx* g = c->g;
    PushHost a{};
    a.fo = fo;
    a.fn = g->buf[g->cur];
    a.n = g->n;
    a.np = c->np;
    push_coeffs(a, n, g->dtau, g->p.expanding, c->p.integrator, c->p.substeps, c->p.interp);
    a.mass = c->mass;
    a.acc = c->acc + 4 * (size_t)(n + 1);
    return a;
}
static bool pushed_at(const cpic_ctx* c, int n) { return n >= c->first_step && c->np > 0; }
// ensembles that can share a launch: the default kernel (one particle step per field step,
// nearest-grid-point gather)
static bool packable(const cpic_ctx* c) { return c->p.substeps <= 1 && c->p.interp == 0; }
// the counting sort of ensemble c by cell, when it is due after a push
static glasma_status sort_if_due(cpic_ctx* c) {
    glasma_ctx* g = c->g;
    if (c->p.bin_every > 0 && ++c->since_sort >= c->p.bin_every) {
        int* cnt = c->sort_ws;
        int* start = cnt + g->ns;
        int* tot = start + g->ns;
        CK(launch_sort(g->prec, c->P[c->pcur], c->P[c->pcur ^ 1], c->np, (int)g->ns, cnt, start, tot, g->st));
        c->pcur ^= 1;
        c->since_sort = 0;
    }
    return GLASMA_OK;
}

extern "C" glasma_status cpic_push_many(cpic_ctx* const* cs, int32_t n_ctx, int32_t n_steps) {
    if (!cs || n_ctx < 1 || n_steps < 0) return fail(GLASMA_ERR_INVALID, "bad arguments");
    for (int i = 0; i < n_ctx; i++) {
        if (!cs[i]) return fail(GLASMA_ERR_INVALID, "null context");
        if (cs[i]->g != cs[0]->g) return fail(GLASMA_ERR_INVALID, "ensembles bound to different field contexts");
        for (int k = 0; k < i; k++)
            if (cs[k] == cs[i]) return fail(GLASMA_ERR_INVALID, "an ensemble is listed twice");
    }
    glasma_ctx* g = cs[0]->g;
    if (g->step < 1) return fail(GLASMA_ERR_INVALID, "field state not initialised");
    for (int k = 0; k < n_steps; k++) {
        if (g->step + 1 >= cs[0]->acc_rows) return fail(GLASMA_ERR_INVALID, "beyond tau_end");
        const int n = g->step;
        const void* fo = g->buf[g->cur];
        glasma_status s = one_field_step(g);
        if (s != GLASMA_OK) return s;
        // the ensembles on the default kernel share launches (blocks interleaved: each
        // sorted by cell, they gather from the same field lines); the others go alone
        PushHost pa[PUSH_PACK_MAX];
        const PartHost* pp[PUSH_PACK_MAX];
        int np = 0;
        const auto flush = [&]() -> glasma_status {
            if (np == 1) CK(launch_push(g->prec, pa[0], *pp[0], g->st));
            else if (np > 1) CK(launch_push_pack(g->prec, pa, pp, np, g->st));
            np = 0;
            return GLASMA_OK;
        };
        for (int i = 0; i < n_ctx; i++) {
            cpic_ctx* c = cs[i];
            if (!pushed_at(c, n)) continue;
            if (!packable(c)) {
                CK(launch_push(g->prec, push_host(c, n, fo), c->P[c->pcur], g->st));
                continue;
            }
            pa[np] = push_host(c, n, fo);
            pp[np] = &c->P[c->pcur];
            if (++np == PUSH_PACK_MAX && (s = flush()) != GLASMA_OK) return s;
        }
        if ((s = flush()) != GLASMA_OK) return s;
        for (int i = 0; i < n_ctx; i++) {
            if (!pushed_at(cs[i], n)) continue;
            if ((s = sort_if_due(cs[i])) != GLASMA_OK) return s;
        }
    }
    return GLASMA_OK;
}

extern "C" glasma_status cpic_push(cpic_ctx* c, int32_t n_steps) {
    if (!c) return fail(GLASMA_ERR_INVALID, "bad arguments");
    return cpic_push_many(&c, 1, n_steps);
}

extern "C" glasma_status broadening_accumulate(cpic_ctx* c, double* out, int64_t cap, int64_t* n_rows) {
    if (!c || !out || !n_rows) return fail(GLASMA_ERR_INVALID, "null argument");
    glasma_ctx* g = c->g;
    std::vector<double> h((size_t)c->acc_rows * 4);
    CK(cudaMemcpyAsync(h.data(), c->acc, h.size() * 8, cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    const double conv = 1.0 / (g->a_gev * g->a_gev);  // lattice momentum^2 -> GeV^2
    int64_t k = 0;
    for (int r = c->first_step; r <= g->step && r < c->acc_rows; r++) {
        if (k >= cap) return fail(GLASMA_ERR_NOSPACE, "host_out too small");
        double* o = out + 5 * k;
        const double cnt = r == c->first_step ? (double)c->np : h[4 * r + 3];
        o[0] = r * g->dtau * g->a_fm;
        for (int i = 0; i < 3; i++) o[1 + i] = (r == c->first_step || cnt <= 0) ? 0.0 : h[4 * r + i] / cnt * conv;
        o[4] = cnt;
        k++;
    }
    *n_rows = k;
    return GLASMA_OK;
}

// ---------------------------------------------------------------- checkpoints
// A checkpoint blob: this header, then the raw device image of the state (field buffer,
// or particle planes followed by the broadening sums).  The header pins what the image
// depends on, so a blob only loads into a context of the same shape.
struct CkptHeader {
    char magic[8];
    int32_t version, prec, n, np;
    int32_t step, first_step, since_sort, acc_rows;
    double dtau, a_fm, mass;
    int32_t expanding, integrator, substeps, interp;
    int64_t body_bytes;
};
static void ckpt_header(CkptHeader& h, const char* magic, const glasma_ctx* g) {
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, magic, 8);
    h.version = 2;  // 2: field buffers of 64 planes (the plaquette group added)
    h.prec = g->prec;
    h.n = g->n;
    h.dtau = g->dtau;
    h.a_fm = g->a_fm;
    h.expanding = g->p.expanding;
}
static bool ckpt_same_shape(const CkptHeader& a, const CkptHeader& b) {
    return !memcmp(a.magic, b.magic, 8) && a.version == b.version && a.prec == b.prec && a.n == b.n && a.np == b.np &&
           a.acc_rows == b.acc_rows && a.dtau == b.dtau && a.a_fm == b.a_fm && a.mass == b.mass &&
           a.expanding == b.expanding && a.integrator == b.integrator && a.substeps == b.substeps && a.interp == b.interp &&
           a.body_bytes == b.body_bytes;
}

extern "C" int64_t glasma_state_bytes(const glasma_ctx* g) {
    if (!g) return GLASMA_ERR_INVALID;
    return (int64_t)(sizeof(CkptHeader) + field_buf_bytes(&g->p));
}
extern "C" glasma_status glasma_export_state(glasma_ctx* g, void* host, int64_t bytes) {
    if (!g || !host) return fail(GLASMA_ERR_INVALID, "null argument");
    if (g->step < 0) return fail(GLASMA_ERR_INVALID, "state not initialised");
    if (bytes < glasma_state_bytes(g)) return fail(GLASMA_ERR_NOSPACE, "host buffer smaller than glasma_state_bytes");
    CkptHeader h;
    ckpt_header(h, "GLSMFLD1", g);
    h.step = g->step;
    h.body_bytes = (int64_t)field_buf_bytes(&g->p);
    memcpy(host, &h, sizeof(h));
    CK(cudaMemcpyAsync((char*)host + sizeof(h), g->buf[g->cur], (size_t)h.body_bytes, cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    return GLASMA_OK;
}
extern "C" glasma_status glasma_import_state(glasma_ctx* g, const void* host, int64_t bytes) {
    if (!g || !host) return fail(GLASMA_ERR_INVALID, "null argument");
    if (bytes < glasma_state_bytes(g)) return fail(GLASMA_ERR_INVALID, "blob smaller than glasma_state_bytes");
    CkptHeader want, got;
    ckpt_header(want, "GLSMFLD1", g);
    want.body_bytes = (int64_t)field_buf_bytes(&g->p);
    memcpy(&got, host, sizeof(got));
    want.step = got.step;
    if (!ckpt_same_shape(want, got) || got.step < 0 || got.step > g->n_steps)
        return fail(GLASMA_ERR_INVALID, "checkpoint does not match this field context");
    CK(cudaMemcpyAsync(g->buf[0], (const char*)host + sizeof(got), (size_t)got.body_bytes, cudaMemcpyHostToDevice,
                       g->st));
    CK(cudaStreamSynchronize(g->st));
    g->cur = 0;
    g->step = got.step;
    return GLASMA_OK;
}

static CkptHeader cpic_header(const cpic_ctx* c) {
    CkptHeader h;
    ckpt_header(h, "GLSMCPC1", c->g);
    h.np = c->np;
    h.acc_rows = c->acc_rows;
    h.mass = c->mass;
    h.integrator = c->p.integrator;
    h.substeps = c->p.substeps > 1 ? c->p.substeps : 1;
    h.interp = c->p.interp;
    h.body_bytes = (int64_t)(part_bytes(c->np, c->g->prec) + (size_t)c->acc_rows * 4 * 8);
    return h;
}
extern "C" int64_t cpic_state_bytes(const cpic_ctx* c) {
    if (!c) return GLASMA_ERR_INVALID;
    return (int64_t)sizeof(CkptHeader) + cpic_header(c).body_bytes;
}
extern "C" glasma_status cpic_export_state(cpic_ctx* c, void* host, int64_t bytes) {
    if (!c || !host) return fail(GLASMA_ERR_INVALID, "null argument");
    if (bytes < cpic_state_bytes(c)) return fail(GLASMA_ERR_NOSPACE, "host buffer smaller than cpic_state_bytes");
    glasma_ctx* g = c->g;
    CkptHeader h = cpic_header(c);
    h.first_step = c->first_step;
    h.since_sort = c->since_sort;
    memcpy(host, &h, sizeof(h));
    char* body = (char*)host + sizeof(h);
    const size_t pb = part_bytes(c->np, g->prec);
    if (c->np > 0) CK(cudaMemcpyAsync(body, c->P[c->pcur].cell, pb, cudaMemcpyDeviceToHost, g->st));
    CK(cudaMemcpyAsync(body + pb, c->acc, (size_t)c->acc_rows * 4 * 8, cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    return GLASMA_OK;
}
extern "C" glasma_status cpic_import_state(cpic_ctx* c, const void* host, int64_t bytes) {
    if (!c || !host) return fail(GLASMA_ERR_INVALID, "null argument");
    if (bytes < cpic_state_bytes(c)) return fail(GLASMA_ERR_INVALID, "blob smaller than cpic_state_bytes");
    glasma_ctx* g = c->g;
    CkptHeader want = cpic_header(c), got;
    memcpy(&got, host, sizeof(got));
    want.first_step = got.first_step;
    want.since_sort = got.since_sort;
    if (!ckpt_same_shape(want, got) || got.first_step < 1 || got.first_step >= c->acc_rows || got.since_sort < 0)
        return fail(GLASMA_ERR_INVALID, "checkpoint does not match this particle ensemble");
    const char* body = (const char*)host + sizeof(got);
    const size_t pb = part_bytes(c->np, g->prec);
    if (c->np > 0) CK(cudaMemcpyAsync(c->P[0].cell, body, pb, cudaMemcpyHostToDevice, g->st));
    CK(cudaMemcpyAsync(c->acc, body + pb, (size_t)c->acc_rows * 4 * 8, cudaMemcpyHostToDevice, g->st));
    CK(cudaStreamSynchronize(g->st));
    c->pcur = 0;
    c->first_step = got.first_step;
    c->since_sort = got.since_sort;
    return GLASMA_OK;
}

extern "C" glasma_status cpic_casimir_drift(cpic_ctx* c, double out[2]) {
    if (!c || !out) return fail(GLASMA_ERR_INVALID, "null argument");
    glasma_ctx* g = c->g;
    CK(launch_casimir_drift(g->prec, c->P[c->pcur], c->np, c->p.q2, c->p.q3, c->cas, g->st));
    CK(cudaMemcpyAsync(out, c->cas, 16, cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    return GLASMA_OK;
}

// ---------------------------------------------------------------- lattice correlators
struct glasma_corr {
    glasma_ctx* g;
    corr_params p;
    int first_step;  // the first step whose fields enter (as the particles formed then)
    int rows;        // accumulator rows: one per step number
    void* state;     // I, J, W planes
    double* acc;     // [rows][6] FP64 sums
};

static int corr_rows(const glasma_params* gp) { return total_steps(gp) + 2; }

extern "C" int64_t corr_workspace_bytes(const glasma_params* gp) {
    glasma_status s = check_params(gp);
    if (s != GLASMA_OK) return s;
    return (int64_t)(align256(corr_state_bytes(gp->precision == GLASMA_FP32, gp->n)) +
                     align256((size_t)corr_rows(gp) * 6 * 8) + 512);
}

extern "C" glasma_status corr_create(glasma_ctx* g, const corr_params* p, void* ws, int64_t ws_bytes,
                                     glasma_corr** out) {
    if (!g || !p || !out) return fail(GLASMA_ERR_INVALID, "null argument");
    if (!ws || ((uintptr_t)ws & 255)) return fail(GLASMA_ERR_INVALID, "workspace must be non-null, 256-byte aligned");
    if (!(p->tau_start_fm >= 0) || !(p->ox0 >= 0) || !(p->ox0 < 1)) return fail(GLASMA_ERR_INVALID, "bad corr_params");
    if (g->corr) return fail(GLASMA_ERR_INVALID, "the context has a correlator attached already");
    if (g->step < 1) return fail(GLASMA_ERR_INVALID, "field state not initialised");
    if (ws_bytes < corr_workspace_bytes(&g->p)) return fail(GLASMA_ERR_NOSPACE, "workspace too small");
    glasma_corr* c = new (std::nothrow) glasma_corr();
    if (!c) return fail(GLASMA_ERR_INVALID, "host allocation failed");
    c->g = g;
    c->p = *p;
    c->rows = corr_rows(&g->p);
    c->first_step = std::max(g->step, std::max(1, (int)llround(p->tau_start_fm / (g->dtau * g->a_fm))));
    char* b = (char*)ws;
    c->state = b;
    c->acc = (double*)(b + align256(corr_state_bytes(g->prec, g->n)));
    CK(launch_corr_reset(g->prec, c->state, g->n, g->st));
    CK(cudaMemsetAsync(c->acc, 0, (size_t)c->rows * 6 * 8, g->st));
    g->corr = c;
    *out = c;
    return GLASMA_OK;
}

static glasma_status corr_after_step(glasma_ctx* g, const void* fo, const void* fn) {
    glasma_corr* c = g->corr;
    const int n_step = g->step;
    if (n_step < c->first_step || n_step + 1 >= c->rows) return GLASMA_OK;
    const int m = n_step - c->first_step;
    const int k0 = (int)floor(c->p.ox0 + m * g->dtau), k1 = (int)floor(c->p.ox0 + (m + 1) * g->dtau);
    const double te = g->p.expanding ? n_step * g->dtau : 1.0;
    CK(launch_corr_step(g->prec, fo, fn, g->n, te, g->dtau, c->state, k0, k1, c->acc + 6 * (size_t)(n_step + 1),
                        g->st));
    return GLASMA_OK;
}

extern "C" glasma_status corr_table(glasma_corr* c, double* out, int64_t cap, int64_t* n_rows) {
    if (!c || !out || !n_rows) return fail(GLASMA_ERR_INVALID, "null argument");
    glasma_ctx* g = c->g;
    if (!g) return fail(GLASMA_ERR_INVALID, "the field context was destroyed");
    std::vector<double> h((size_t)c->rows * 6);
    CK(cudaMemcpyAsync(h.data(), c->acc, h.size() * 8, cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    const double conv = 1.0 / (g->a_gev * g->a_gev) / ((double)g->n * g->n);  // site mean, lattice -> GeV^2
    int64_t k = 0;
    for (int r = c->first_step; r <= g->step && r < c->rows; r++) {
        if (k >= cap) return fail(GLASMA_ERR_NOSPACE, "host_out too small");
        double* o = out + 7 * k;
        o[0] = r * g->dtau * g->a_fm;
        for (int i = 0; i < 6; i++) o[1 + i] = r == c->first_step ? 0.0 : h[6 * (size_t)r + i] * conv;
        k++;
    }
    *n_rows = k;
    return GLASMA_OK;
}

static void corr_detach(glasma_ctx* g) {
    if (g->corr) g->corr->g = nullptr;
    g->corr = nullptr;
}

extern "C" void corr_destroy(glasma_corr* c) {
    if (!c) return;
    if (c->g && c->g->corr == c) c->g->corr = nullptr;
    delete c;
}
