// Many Glasma events of uneven lattice sizes, each with its own particle
// ensemble, advanced together (the event average of Sec. 2, "Quantifying the
// effect of Glasma", of arXiv:2307.07999 taken over independent events).
//
// Events are ordered by their step count (descending); iteration k advances
// every event whose step k+1 is below its own n_steps, so the active events,
// their field tiles and their particle blocks are always prefixes of fixed
// tables.  The per-step arguments (tau-dependent coefficients, ping-pong
// buffers, accumulator rows) are precomputed per iteration, so one run is a
// fixed sequence of launches that is captured once into a CUDA graph.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "../../include/glasma.h"
#include "batch.h"
#include "internal.h"

using namespace glasma;

static thread_local char b_err[512] = "";
const char* glasma_batch_error() { return b_err; }

static glasma_status bfail(glasma_status s, const char* msg) {
    snprintf(b_err, sizeof(b_err), "%s", msg);
    glasma_set_error(b_err);
    return s;
}
static glasma_status bcuda(cudaError_t e, const char* where) {
    snprintf(b_err, sizeof(b_err), "%s: %s", where, cudaGetErrorString(e));
    glasma_set_error(b_err);
    return GLASMA_ERR_CUDA;
}
#define BCK(call)                                          \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return bcuda(e_, #call);    \
    } while (0)

static const double HBARC_B = 0.1973269804;

static int steps_of(const glasma_params& p) {
    const double a_fm = p.L_fm / p.n;
    return (int)ceil(p.tau_end_fm / (p.dtau_over_a * a_fm) - 1e-9);
}
static size_t fbytes(const glasma_params& p) {
    return align256((size_t)N_FIELD_PLANES * (size_t)p.n * p.n * (p.precision ? 4 : 8));
}

struct Layout {
    size_t fields, parts, accs, tables, scratch, total;
};

static Layout layout(const glasma_params* ev, const cpic_params* pp, int E, size_t fft_work) {
    Layout L{};
    int nmax = 0, smax = 0;
    size_t npmax = 0;
    for (int e = 0; e < E; e++) {
        L.fields += 4 * fbytes(ev[e]);
        const size_t ns = (size_t)ev[e].n * ev[e].n;
        L.fields += align256(ns * record_bytes(ev[e].precision)) + align256(ns * 4);
        L.parts += 2 * part_bytes(pp[e].n_particles, ev[e].precision);
        L.parts += 6 * align256((size_t)pp[e].n_particles * (ev[e].precision ? 4 : 8)) + 256;
        L.accs += align256(((size_t)steps_of(ev[e]) + 2) * 4 * 8);
        nmax = std::max(nmax, ev[e].n);
        smax = std::max(smax, steps_of(ev[e]));
        npmax = std::max(npmax, (size_t)pp[e].n_particles);
    }
    const int prec = ev[0].precision;
    L.tables = align256((size_t)smax * E * step_args_size(prec)) + align256((size_t)smax * E * push_args_size(prec)) +
               3 * align256((size_t)4 << 20) + align256(256 + ((size_t)smax + 2) * 8 + ((size_t)E + 1) * 8);
    const size_t ic = ic_scratch_bytes(nmax, fft_work);
    const size_t srt = align256(sort_scratch_ints(nmax * nmax) * 4);
    L.scratch = std::max(ic, srt) + 256;
    L.total = L.fields + L.parts + L.accs + L.tables + L.scratch + 16 * 256 * (size_t)E + 4096;
    return L;
}

static glasma_status check_batch(const glasma_params* ev, const cpic_params* pp, int E) {
    if (!ev || !pp || E < 1 || E > 65536) return bfail(GLASMA_ERR_INVALID, "bad event list");
    for (int e = 0; e < E; e++) {
        if (ev[e].precision != ev[0].precision || ev[e].expanding != 1)
            return bfail(GLASMA_ERR_INVALID, "all events need the same precision and the expanding evolution");
        if (ev[e].n < 2 || ev[e].n > 16384 || !(ev[e].L_fm > 0) || !(ev[e].dtau_over_a > 0) || ev[e].dtau_over_a > 1 ||
            ev[e].n_sheets < 1 || !(ev[e].tau_end_fm > 0))
            return bfail(GLASMA_ERR_INVALID, "bad event parameters");
        if (pp[e].n_particles < 0 || pp[e].mass_GeV < 0 || pp[e].tau_form_fm < 0 || pp[e].p_max_GeV < pp[e].p_min_GeV ||
            (pp[e].init_kind != 0 && pp[e].init_kind != 1) || (pp[e].integrator != 0 && pp[e].integrator != 1) ||
            pp[e].substeps < 0 || pp[e].substeps > 64 || (pp[e].interp != 0 && pp[e].interp != 1))
            return bfail(GLASMA_ERR_INVALID, "bad particle parameters");
    }
    return GLASMA_OK;
}

extern "C" int64_t glasma_batch_workspace_bytes(const glasma_params* ev, const cpic_params* pp, int32_t E) {
    glasma_status s = check_batch(ev, pp, E);
    if (s != GLASMA_OK) return s;
    int nmax = 0;
    for (int e = 0; e < E; e++) nmax = std::max(nmax, ev[e].n);
    const char* err = "";
    const size_t work = ic_fft_work_bytes(nmax, &err);
    if (work == (size_t)-1) return bfail(GLASMA_ERR_CUDA, err);
    return (int64_t)layout(ev, pp, E, work).total;
}

struct Arena2 {
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

extern "C" glasma_status glasma_batch_create(const glasma_params* ev, const cpic_params* pp, int32_t E, void* ws,
                                             int64_t ws_bytes, void* stream, glasma_batch** out) {
    glasma_status s = check_batch(ev, pp, E);
    if (s != GLASMA_OK) return s;
    if (!ws || !out || ((uintptr_t)ws & 255)) return bfail(GLASMA_ERR_INVALID, "workspace must be non-null, 256-byte aligned");
    const int64_t need = glasma_batch_workspace_bytes(ev, pp, E);
    if (need < 0) return (glasma_status)need;
    if (ws_bytes < need) return bfail(GLASMA_ERR_NOSPACE, "workspace too small");
    glasma_batch* b = new (std::nothrow) glasma_batch();
    if (!b) return bfail(GLASMA_ERR_INVALID, "host allocation failed");
    b->prec = ev[0].precision;
    b->st = (cudaStream_t)stream;
    b->E = E;
    int nmax = 0;
    for (int e = 0; e < E; e++) nmax = std::max(nmax, ev[e].n);
    const char* err = "";
    b->fft_work = ic_fft_work_bytes(nmax, &err);
    b->nmax = nmax;
    // order: step count descending (stable), so active events are prefixes
    std::vector<int> ord(E);
    for (int e = 0; e < E; e++) ord[e] = e;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int c) { return steps_of(ev[a]) > steps_of(ev[c]); });
    b->pos.assign(E, 0);
    Arena2 A{(char*)ws, (size_t)ws_bytes, 0};
    b->ev.resize(E);
    for (int i = 0; i < E; i++) {
        const int e = ord[i];
        b->pos[e] = i;
        BatchEvent& x = b->ev[i];
        x.gp = ev[e];
        x.pp = pp[e];
        x.id = e;
        x.n = ev[e].n;
        x.ns = (size_t)x.n * x.n;
        x.n_steps = steps_of(ev[e]);
        x.a_fm = ev[e].L_fm / x.n;
        x.a_gev = x.a_fm / HBARC_B;
        x.dtau = ev[e].dtau_over_a;
        x.np = pp[e].n_particles;
        x.n_form = std::max(1, (int)lround(pp[e].tau_form_fm / (x.dtau * x.a_fm)));
        x.mass = pp[e].mass_GeV * x.a_gev;
        if (pp[e].substeps > 1 || pp[e].interp) b->any_sub = true;
        x.buf[0] = A.take(fbytes(ev[e]));
        x.buf[1] = A.take(fbytes(ev[e]));
        x.buf[2] = A.take(fbytes(ev[e]));
        x.init_buf = A.take(fbytes(ev[e]));
        x.rec = A.take(x.ns * record_bytes(b->prec));
        x.occ = (int*)A.take(x.ns * 4);
        const size_t pb = part_bytes(x.np, b->prec);
        x.part_bytes = pb;
        x.part_base = A.take(pb);
        x.part_init = A.take(pb);
        x.P = part_layout(x.part_base, x.np, b->prec);
        x.frc = A.take(6 * x.P.pstride * (b->prec ? 4 : 8));
        x.acc_rows = x.n_steps + 2;
        x.acc = (double*)A.take((size_t)x.acc_rows * 4 * 8);
        x.mon = (double*)A.take(256);
        if (!x.buf[0] || !x.buf[1] || !x.buf[2] || !x.init_buf || !x.rec || !x.occ || !x.frc || !x.part_base || !x.part_init || !x.acc || !x.mon) {
            delete b;
            return bfail(GLASMA_ERR_NOSPACE, "workspace too small");
        }
    }
    b->max_iter = 0;
    for (auto& x : b->ev) b->max_iter = std::max(b->max_iter, x.n_steps - 1);
    b->step_args = A.take(align256((size_t)std::max(1, b->max_iter) * E * step_args_size(b->prec)));
    b->push_args = A.take(align256((size_t)std::max(1, b->max_iter) * E * push_args_size(b->prec)));
    b->tiles_dev = A.take((size_t)4 << 20);
    b->gtiles_dev = A.take((size_t)4 << 20);
    b->pitems_dev = A.take((size_t)4 << 20);
    b->scratch = A.take(std::max(ic_scratch_bytes(nmax, b->fft_work), align256(sort_scratch_ints(nmax * nmax) * 4)));
    b->pers_ctrl = A.take(256 + ((size_t)std::max(1, b->max_iter) + 2) * 8 + ((size_t)E + 1) * 8);
    if (!b->step_args || !b->push_args || !b->tiles_dev || !b->gtiles_dev || !b->pitems_dev || !b->scratch ||
        !b->pers_ctrl) {
        delete b;
        return bfail(GLASMA_ERR_NOSPACE, "workspace too small");
    }
    // the persistent kernel's counters and error word start cleared (the workspace is
    // the caller's uninitialised memory)
    if (cudaMemsetAsync(b->pers_ctrl, 0, 256, b->st) != cudaSuccess || cudaStreamSynchronize(b->st) != cudaSuccess) {
        delete b;
        return bfail(GLASMA_ERR_CUDA, "clearing the persistent control block failed");
    }
    *out = b;
    return GLASMA_OK;
}

// tile items of the chosen field variant, grouped by event
static glasma_status build_gtiles(glasma_batch* b) {
    int tx, ty, mb;
    field_variant_shape(b->prec, b->fvar, &tx, &ty, &mb);
    std::vector<TileItemH> tiles;
    b->gtiles_upto.assign(b->E + 1, 0);
    for (int i = 0; i < b->E; i++) {
        const BatchEvent& x = b->ev[i];
        for (int y0 = 0; y0 < x.n; y0 += ty)
            for (int x0 = 0; x0 < x.n; x0 += tx) tiles.push_back({i, x0, y0});
        b->gtiles_upto[i + 1] = (int)tiles.size();
    }
    if (tiles.size() * sizeof(TileItemH) > ((size_t)4 << 20)) return bfail(GLASMA_ERR_NOSPACE, "tile table exceeds its reserve");
    BCK(cudaMemcpyAsync(b->gtiles_dev, tiles.data(), tiles.size() * sizeof(TileItemH), cudaMemcpyHostToDevice, b->st));
    BCK(cudaStreamSynchronize(b->st));  // the host vector goes out of scope
    return GLASMA_OK;
}

// tables of per-iteration arguments, tile items and particle-block items
static glasma_status build_tables(glasma_batch* b) {
    const int E = b->E, K = std::max(1, b->max_iter);
    const int tx = field_tile_x(b->prec), ty = field_tile_y(b->prec);
    std::vector<TileItemH> tiles;
    std::vector<PushItemH> pits;
    b->tiles_upto.assign(E + 1, 0);
    b->pitems_upto.assign(E + 1, 0);
    for (int i = 0; i < E; i++) {
        const BatchEvent& x = b->ev[i];
        for (int y0 = 0; y0 < x.n; y0 += ty)
            for (int x0 = 0; x0 < x.n; x0 += tx) tiles.push_back({i, x0, y0});
        for (int j0 = 0; j0 < x.np; j0 += 256) pits.push_back({i, j0});
        b->tiles_upto[i + 1] = (int)tiles.size();
        b->pitems_upto[i + 1] = (int)pits.size();
    }
    if (tiles.size() * sizeof(TileItemH) > ((size_t)4 << 20) || pits.size() * sizeof(PushItemH) > ((size_t)4 << 20))
        return bfail(GLASMA_ERR_NOSPACE, "item tables exceed their reserve");
    BCK(cudaMemcpyAsync(b->tiles_dev, tiles.data(), tiles.size() * sizeof(TileItemH), cudaMemcpyHostToDevice, b->st));
    BCK(prepare_field_variants(b->prec));
    BCK(prepare_push_staged());
    {
        glasma_status gs = build_gtiles(b);
        if (gs != GLASMA_OK) return gs;
    }
    BCK(cudaMemcpyAsync(b->pitems_dev, pits.data(), pits.size() * sizeof(PushItemH), cudaMemcpyHostToDevice, b->st));
    const size_t sa = step_args_size(b->prec), pa = push_args_size(b->prec);
    std::vector<char> hs((size_t)K * E * sa, 0), hp((size_t)K * E * pa, 0);
    b->active.assign(K, 0);
    for (int k = 0; k < K; k++) {
        const int s = k + 1;  // every event starts at step 1
        int act = 0;
        for (int i = 0; i < E; i++) {
            const BatchEvent& x = b->ev[i];
            const bool on = s < x.n_steps;
            if (on) act = i + 1;
            const void* src = x.buf[k % 3];
            void* dst = x.buf[(k + 1) % 3];
            const int reunit = reunit_code(x.gp.reunit_every, s);
            StepHost st = step_coeffs(src, dst, x.n, s, x.dtau, 1, reunit);
            // the batched pushes form the clover themselves (the batched field kernels
            // store no plaquettes; the per-event mode's one-event kernels do)
            st.plaq = nullptr;
            // gather records (used by the REC field kernels of the record push): at the
            // particles' first step every cell gets one, later the cells stamped by the push
            st.rec = x.rec;
            st.occ = x.occ;
            st.all_rec = s == x.n_form ? 1 : 0;
            pack_step_args(b->prec, st, hs.data() + ((size_t)k * E + i) * sa);
            PushHost ph{};
            ph.fo = src; ph.fn = dst; ph.n = x.n; ph.np = x.np;
            push_coeffs(ph, s, x.dtau, 1, x.pp.integrator, x.pp.substeps, x.pp.interp);
            ph.mass = x.mass;
            ph.acc = (on && s >= x.n_form) ? x.acc + 4 * (size_t)(s + 1) : nullptr;
            ph.rec = x.rec;
            ph.occ = x.occ;
            ph.epoch_next = s + 1;
            ph.frc = x.frc;
            pack_push_args(b->prec, ph, x.P, hp.data() + ((size_t)k * E + i) * pa);
        }
        b->active[k] = act;
    }
    // first launch outside any stream capture sets the kernels' shared-memory attribute
    BCK(launch_field_step_batched(b->prec, nullptr, nullptr, 0, b->st));
    {
        // persistent-kernel control block: 256 B of counters, then work counters [K + 1],
        // active [K], tiles_upto [E + 1], pitems_upto [E + 1]
        std::vector<int> h(((size_t)K + 1) + K + 2 * ((size_t)E + 1), 0);
        int* w = h.data();
        for (int k = 0; k < K; k++) w[(K + 1) + k] = b->active[k];
        for (int i = 0; i <= E; i++) {
            w[(K + 1) + K + i] = b->tiles_upto[i];
            w[(K + 1) + K + (E + 1) + i] = b->pitems_upto[i];
        }
        BCK(cudaMemcpyAsync((char*)b->pers_ctrl + 256, h.data(), h.size() * 4, cudaMemcpyHostToDevice, b->st));
    }
    BCK(cudaMemcpyAsync(b->step_args, hs.data(), hs.size(), cudaMemcpyHostToDevice, b->st));
    BCK(cudaMemcpyAsync(b->push_args, hp.data(), hp.size(), cudaMemcpyHostToDevice, b->st));
    BCK(cudaStreamSynchronize(b->st));
    return GLASMA_OK;
}

extern "C" glasma_status glasma_batch_init(glasma_batch* b, int64_t* ic_failures) {
    if (!b) return bfail(GLASMA_ERR_INVALID, "null batch");
    long long fails_total = 0;
    for (auto& x : b->ev) {
        const ICScratch sc = ic_layout(b->scratch, x.n, b->fft_work);
        const char* err = "";
        long long f = 0;
        double m = 0;
        int mx = 0;
        const int it = x.gp.newton_max_iter > 0 ? x.gp.newton_max_iter : 100;
        const double tol = x.gp.newton_tol > 0 ? x.gp.newton_tol : 1e-12;
        int rc = ic_run(b->prec, x.n, x.gp.n_sheets, x.gp.g2mu_GeV * x.a_gev, x.gp.m_ir_GeV * x.a_gev, x.gp.seed, x.dtau,
                        tol, it, sc, x.init_buf, b->st, &f, &m, &mx, &err);
        if (rc == -6) return bfail(GLASMA_ERR_NOSPACE, err);
        if (rc != 0) return bfail(GLASMA_ERR_CUDA, err);
        x.ic_fails = f;
        x.ic_mean = m;
        x.ic_max = mx;
        fails_total += f;
        // particles: Philox state, then sorted by cell once (gather locality)
        PartHost tmp = part_layout(x.part_base, x.np, b->prec);
        BCK(launch_part_init(b->prec, tmp, x.np, x.n, x.pp.init_kind, x.pp.p_min_GeV * x.a_gev,
                             x.pp.p_max_GeV * x.a_gev, x.pp.q2, x.pp.q3, x.pp.seed, x.mass, b->st));
        const PartHost dst = part_layout(x.part_init, x.np, b->prec);
        int* cnt = (int*)b->scratch;
        int* start = cnt + x.ns;
        int* tot = start + x.ns;
        BCK(launch_sort(b->prec, tmp, dst, x.np, (int)x.ns, cnt, start, tot, b->st));
        BCK(cudaStreamSynchronize(b->st));
    }
    if (ic_failures) *ic_failures = fails_total;
    glasma_status s = build_tables(b);
    if (s != GLASMA_OK) return s;
    b->initialised = true;
    b->graph_ready = false;
    return GLASMA_OK;
}

// restore every event to its initial state (step 1, particles at formation)
static cudaError_t enqueue_restore(glasma_batch* b) {
    for (auto& x : b->ev) {
        cudaError_t e = cudaMemcpyAsync(x.buf[0], x.init_buf, fbytes(x.gp), cudaMemcpyDeviceToDevice, b->st);
        if (e != cudaSuccess) return e;
        e = cudaMemcpyAsync(x.part_base, x.part_init, x.part_bytes, cudaMemcpyDeviceToDevice, b->st);
        if (e != cudaSuccess) return e;
        e = cudaMemsetAsync(x.acc, 0, (size_t)x.acc_rows * 4 * 8, b->st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// the graph and eager modes run the record push (and the field kernels that write its
// records) when it is the chosen push kernel and no event needs the sub-stepped push
static bool batch_records(const glasma_batch* b) { return !b->any_sub && b->pvar == PUSH_VARIANT_RECORD; }

static cudaError_t enqueue_batched(glasma_batch* b) {
    cudaError_t e = enqueue_restore(b);
    if (e != cudaSuccess) return e;
    const size_t sa = step_args_size(b->prec), pa = push_args_size(b->prec);
    // record push: field launch k writes the records push k reads, and push k stamps the
    // cells field launch k+1 writes records for, so both stay on one stream
    const bool rec = batch_records(b);
    const bool two = !rec && b->two_streams && b->st2 != nullptr;
    cudaStream_t sp = two ? b->st2 : b->st;  // the stream of the pushes
    const int K = b->max_iter;
    if (two) {  // the pushes see the restore
        e = cudaEventRecord(b->sev[2 * (size_t)K], b->st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->st2, b->sev[2 * (size_t)K], 0);
        if (e != cudaSuccess) return e;
    }
    int last_push = -1;
    b->tev_used = 0;
    for (int k = 0; k < b->max_iter; k++) {
        const int act = b->active[k];
        if (act == 0) break;
        if (two && k >= 2) {  // field k overwrites the buffer push k-2 reads
            e = cudaStreamWaitEvent(b->st, b->sev[2 * (size_t)(k - 2) + 1], 0);
            if (e != cudaSuccess) return e;
        }
        // (timing: external event records, so that a captured graph keeps them as nodes)
        if (b->timing) {
            e = cudaEventRecordWithFlags(b->tev[2 * k], b->st, cudaEventRecordExternal);
            if (e != cudaSuccess) return e;
        }
        e = launch_field_step_variant(b->prec, b->fvar, (char*)b->step_args + (size_t)k * b->E * sa, b->gtiles_dev,
                                      b->gtiles_upto[act], b->st, rec);
        if (e != cudaSuccess) return e;
        if (b->timing) {
            e = cudaEventRecordWithFlags(b->tev[2 * k + 1], b->st, cudaEventRecordExternal);
            if (e != cudaSuccess) return e;
            b->tev_used = k + 1;
        }
        if (two) {
            e = cudaEventRecord(b->sev[2 * (size_t)k], b->st);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(sp, b->sev[2 * (size_t)k], 0);
            if (e != cudaSuccess) return e;
        }
        e = launch_push_batched(b->prec, b->any_sub ? PUSH_VARIANT_SUB : b->pvar, (char*)b->push_args + (size_t)k * b->E * pa, b->pitems_dev,
                                b->pitems_upto[act], sp);
        if (e != cudaSuccess) return e;
        if (two) {
            e = cudaEventRecord(b->sev[2 * (size_t)k + 1], sp);
            if (e != cudaSuccess) return e;
            last_push = k;
        }
    }
    if (two && last_push >= 0) {  // join: the run ends with its last push
        e = cudaStreamWaitEvent(b->st, b->sev[2 * (size_t)last_push + 1], 0);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static cudaError_t enqueue_per_event(glasma_batch* b) {
    cudaError_t e = enqueue_restore(b);
    if (e != cudaSuccess) return e;
    for (auto& x : b->ev) {
        for (int s = 1; s < x.n_steps; s++) {
            const int k = s - 1;
            const StepHost st = step_coeffs(x.buf[k % 3], x.buf[(k + 1) % 3], x.n, s, x.dtau, 1,
                                            reunit_code(x.gp.reunit_every, s));
            e = launch_field_step(b->prec, st, b->st);
            if (e != cudaSuccess) return e;
            if (s >= x.n_form && x.np > 0) {
                PushHost ph{};
                ph.fo = x.buf[k % 3]; ph.fn = x.buf[(k + 1) % 3]; ph.n = x.n; ph.np = x.np;
                push_coeffs(ph, s, x.dtau, 1, x.pp.integrator, x.pp.substeps, x.pp.interp);
                ph.mass = x.mass;
                ph.acc = x.acc + 4 * (size_t)(s + 1);
                e = launch_push(b->prec, ph, x.P, b->st);
                if (e != cudaSuccess) return e;
            }
        }
    }
    return cudaSuccess;
}

static glasma_status run_graph(glasma_batch* b) {
    if (b->st == nullptr || b->st == cudaStreamLegacy || b->st == cudaStreamPerThread)
        return bfail(GLASMA_ERR_INVALID, "graph mode needs a created stream (the default stream cannot be captured)");
    cudaGraphExec_t& exec = b->exec;
    bool& ready = b->graph_ready;
    if (!ready) {
        cudaGraph_t g = nullptr;
        BCK(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = enqueue_batched(b);
        cudaError_t e2 = cudaStreamEndCapture(b->st, &g);  // always end the capture
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return bcuda(e != cudaSuccess ? e : e2, "graph capture");
        }
        cudaError_t e3 = cudaGraphInstantiate(&exec, g, 0);
        cudaGraphDestroy(g);
        BCK(e3);
        ready = true;
    }
    BCK(cudaGraphLaunch(exec, b->st));
    return GLASMA_OK;
}

extern "C" glasma_status glasma_batch_run(glasma_batch* b, int32_t mode) {
    if (!b || !b->initialised) return bfail(GLASMA_ERR_INVALID, "batch not initialised");
    switch (mode) {
        case GLASMA_BATCH_PER_EVENT: BCK(enqueue_per_event(b)); return GLASMA_OK;
        case GLASMA_BATCH_EAGER: BCK(enqueue_batched(b)); return GLASMA_OK;
        case GLASMA_BATCH_PERSISTENT:
            if (b->any_sub) return bfail(GLASMA_ERR_INVALID, "the persistent mode does not take sub-stepped or cloud-in-cell particles");
            return batch_run_persistent(b);
        case GLASMA_BATCH_GRAPH: return run_graph(b);
        default: return bfail(GLASMA_ERR_INVALID, "unknown mode");
    }
}

extern "C" glasma_status glasma_batch_broadening(glasma_batch* b, int32_t event, double* out, int64_t cap,
                                                 int64_t* n_rows) {
    if (!b || !out || !n_rows || event < 0 || event >= b->E) return bfail(GLASMA_ERR_INVALID, "bad arguments");
    const BatchEvent& x = b->ev[b->pos[event]];
    std::vector<double> h((size_t)x.acc_rows * 4);
    BCK(cudaMemcpyAsync(h.data(), x.acc, h.size() * 8, cudaMemcpyDeviceToHost, b->st));
    BCK(cudaStreamSynchronize(b->st));
    if (batch_timed_out(b)) return bfail(GLASMA_ERR_TIMEOUT, "persistent kernel: a grid barrier wait ran out");
    const double conv = 1.0 / (x.a_gev * x.a_gev);
    int64_t k = 0;
    for (int r = x.n_form; r <= x.n_steps && r < x.acc_rows; r++) {
        if (k >= cap) return bfail(GLASMA_ERR_NOSPACE, "host_out too small");
        double* o = out + 5 * k;
        const double cnt = r == x.n_form ? (double)x.np : h[4 * r + 3];
        o[0] = r * x.dtau * x.a_fm;
        for (int i = 0; i < 3; i++) o[1 + i] = (r == x.n_form || cnt <= 0) ? 0.0 : h[4 * r + i] / cnt * conv;
        o[4] = cnt;
        k++;
    }
    *n_rows = k;
    return GLASMA_OK;
}

extern "C" glasma_status glasma_batch_work(const glasma_batch* b, int64_t* site_updates, int64_t* particle_steps) {
    if (!b) return bfail(GLASMA_ERR_INVALID, "null batch");
    int64_t su = 0, ps = 0;
    for (const auto& x : b->ev) {
        su += (int64_t)x.ns * (x.n_steps - 1);
        ps += (int64_t)x.np * std::max(0, x.n_steps - x.n_form);
    }
    if (site_updates) *site_updates = su;
    if (particle_steps) *particle_steps = ps;
    return GLASMA_OK;
}

extern "C" glasma_status glasma_batch_diagnostics(glasma_batch* b, int32_t event, double out[8]) {
    if (!b || !out || event < 0 || event >= b->E) return bfail(GLASMA_ERR_INVALID, "bad arguments");
    const BatchEvent& x = b->ev[b->pos[event]];
    const int last = x.n_steps;  // final state at step n_steps sits in buf[(n_steps - 1) % 3]
    BCK(launch_monitors(b->prec, x.buf[(last - 1) % 3], x.n, last * x.dtau, x.mon, b->st));
    double m[8];
    BCK(cudaMemcpyAsync(m, x.mon, sizeof(m), cudaMemcpyDeviceToHost, b->st));
    BCK(cudaStreamSynchronize(b->st));
    const double ns = (double)x.ns;
    out[0] = m[1] > 0 ? sqrt(m[0] / m[1]) : sqrt(m[0]);
    out[1] = m[2] / ns;
    out[2] = m[3] / ns;
    out[3] = m[4] / ns;
    out[4] = m[5] / ns;
    out[5] = m[6];
    out[6] = last * x.dtau;
    out[7] = m[7];
    return GLASMA_OK;
}

// raw device-layout initial state of all events (fields + particles), in event order
extern "C" int64_t glasma_batch_state_bytes(const glasma_batch* b) {
    if (!b) return GLASMA_ERR_INVALID;
    size_t t = 0;
    for (const auto& x : b->ev) t += fbytes(x.gp) + x.part_bytes;
    return (int64_t)t;
}
extern "C" glasma_status glasma_batch_export_state(glasma_batch* b, void* host, int64_t bytes) {
    if (!b || !host || bytes < glasma_batch_state_bytes(b)) return bfail(GLASMA_ERR_INVALID, "bad arguments");
    char* h = (char*)host;
    for (const auto& x : b->ev) {
        BCK(cudaMemcpyAsync(h, x.init_buf, fbytes(x.gp), cudaMemcpyDeviceToHost, b->st));
        h += fbytes(x.gp);
        BCK(cudaMemcpyAsync(h, x.part_init, x.part_bytes, cudaMemcpyDeviceToHost, b->st));
        h += x.part_bytes;
    }
    BCK(cudaStreamSynchronize(b->st));
    return GLASMA_OK;
}
extern "C" glasma_status glasma_batch_import_state(glasma_batch* b, const void* host, int64_t bytes) {
    if (!b || !host || bytes < glasma_batch_state_bytes(b)) return bfail(GLASMA_ERR_INVALID, "bad arguments");
    if (!b->initialised) return bfail(GLASMA_ERR_INVALID, "batch not initialised");
    const char* h = (const char*)host;  // host memory, or device memory staged by the caller
    for (auto& x : b->ev) {
        BCK(cudaMemcpyAsync(x.init_buf, h, fbytes(x.gp), cudaMemcpyDefault, b->st));
        h += fbytes(x.gp);
        BCK(cudaMemcpyAsync(x.part_init, h, x.part_bytes, cudaMemcpyDefault, b->st));
        h += x.part_bytes;
    }
    return GLASMA_OK;
}

// one eager run of the graph mode's launches with CUDA events around every launch (on the
// batch stream): the batched field kernel is the main kernel, the push the other
extern "C" glasma_status glasma_batch_profile(glasma_batch* b, int32_t mode, double* main_ms, int64_t* main_launches,
                                              int64_t* main_sites, int64_t* main_particle_steps, double* other_ms) {
    if (!b || !b->initialised) return bfail(GLASMA_ERR_INVALID, "batch not initialised");
    (void)mode;
    BCK(enqueue_restore(b));
    const size_t sa = step_args_size(b->prec), pa = push_args_size(b->prec);
    const int K = b->max_iter;
    std::vector<cudaEvent_t> ev(4 * (size_t)K);
    for (auto& e : ev) BCK(cudaEventCreate(&e));
    int64_t sites = 0;
    int used = 0;
    for (int k = 0; k < K; k++) {
        const int act = b->active[k];
        if (act == 0) break;
        for (int i = 0; i < act; i++) sites += (int64_t)b->ev[i].ns;
        const void* sargs = (char*)b->step_args + (size_t)k * b->E * sa;
        const void* pargs = (char*)b->push_args + (size_t)k * b->E * pa;
        BCK(cudaEventRecord(ev[4 * k + 0], b->st));
        BCK(launch_field_step_variant(b->prec, b->fvar, sargs, b->gtiles_dev, b->gtiles_upto[act], b->st,
                                      batch_records(b)));
        BCK(cudaEventRecord(ev[4 * k + 1], b->st));
        BCK(cudaEventRecord(ev[4 * k + 2], b->st));
        BCK(launch_push_batched(b->prec, b->any_sub ? PUSH_VARIANT_SUB : b->pvar, pargs, b->pitems_dev,
                                b->pitems_upto[act], b->st));
        BCK(cudaEventRecord(ev[4 * k + 3], b->st));
        used = k + 1;
    }
    BCK(cudaStreamSynchronize(b->st));
    double mm = 0, om = 0;
    for (int k = 0; k < used; k++) {
        float a = 0, c = 0;
        BCK(cudaEventElapsedTime(&a, ev[4 * k + 0], ev[4 * k + 1]));
        BCK(cudaEventElapsedTime(&c, ev[4 * k + 2], ev[4 * k + 3]));
        mm += a;
        om += c;
    }
    for (auto& e : ev) cudaEventDestroy(e);
    if (main_ms) *main_ms = mm;
    if (main_launches) *main_launches = used;
    if (main_sites) *main_sites = sites;
    if (main_particle_steps) *main_particle_steps = 0;
    if (other_ms) *other_ms = om;
    return GLASMA_OK;
}

extern "C" int32_t glasma_field_tile_variants(int32_t precision) {
    return field_variants(precision == GLASMA_FP64 ? 0 : 1);
}
extern "C" glasma_status glasma_field_tile_shape(int32_t precision, int32_t v, int32_t* tx, int32_t* ty,
                                                 int32_t* min_ctas) {
    const int prec = precision == GLASMA_FP64 ? 0 : 1;
    if (v < 0 || v >= field_variants(prec) || !tx || !ty || !min_ctas) return bfail(GLASMA_ERR_INVALID, "bad arguments");
    int a, c, m;
    field_variant_shape(prec, v, &a, &c, &m);
    *tx = a; *ty = c; *min_ctas = m;
    return GLASMA_OK;
}
extern "C" int32_t glasma_batch_variant(const glasma_batch* b) { return b ? b->fvar : GLASMA_ERR_INVALID; }
extern "C" glasma_status glasma_batch_set_variant(glasma_batch* b, int32_t v) {
    if (!b || !b->initialised) return bfail(GLASMA_ERR_INVALID, "batch not initialised");
    if (v < 0 || v >= field_variants(b->prec)) return bfail(GLASMA_ERR_INVALID, "no such tile variant");
    if (v == b->fvar) return GLASMA_OK;
    b->fvar = v;
    if (b->graph_ready) {
        cudaGraphExecDestroy(b->exec);
        b->graph_ready = false;
    }
    return build_gtiles(b);
}
extern "C" glasma_status glasma_batch_set_push_stream(glasma_batch* b, int32_t separate) {
    if (!b || !b->initialised) return bfail(GLASMA_ERR_INVALID, "batch not initialised");
    if ((separate != 0) == b->two_streams) return GLASMA_OK;
    if (separate && !b->st2) {
        BCK(cudaStreamCreateWithFlags(&b->st2, cudaStreamNonBlocking));
        b->sev.assign(2 * (size_t)std::max(1, b->max_iter) + 1, nullptr);
        for (auto& e : b->sev) BCK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    b->two_streams = separate != 0;
    if (b->graph_ready) {  // captured again with (or without) the second stream
        cudaGraphExecDestroy(b->exec);
        b->graph_ready = false;
    }
    return GLASMA_OK;
}
extern "C" glasma_status glasma_batch_set_graph_timing(glasma_batch* b, int32_t on) {
    if (!b || !b->initialised) return bfail(GLASMA_ERR_INVALID, "batch not initialised");
    if ((on != 0) == b->timing) return GLASMA_OK;
    if (on && b->tev.empty()) {
        b->tev.assign(2 * (size_t)std::max(1, b->max_iter), nullptr);
        for (auto& e : b->tev) BCK(cudaEventCreate(&e));
    }
    b->timing = on != 0;
    if (b->graph_ready) {  // captured again with (or without) the event nodes
        cudaGraphExecDestroy(b->exec);
        b->graph_ready = false;
    }
    return GLASMA_OK;
}
extern "C" glasma_status glasma_batch_graph_times(glasma_batch* b, double* field_ms, int64_t* launches,
                                                  double* span_ms) {
    if (!b || !field_ms || !launches || !span_ms) return bfail(GLASMA_ERR_INVALID, "null argument");
    if (!b->timing || b->tev_used == 0) return bfail(GLASMA_ERR_INVALID, "no timed run (set graph timing, then run)");
    BCK(cudaEventSynchronize(b->tev[2 * (size_t)b->tev_used - 1]));
    double t = 0.0;
    for (int k = 0; k < b->tev_used; k++) {
        float ms = 0.f;
        BCK(cudaEventElapsedTime(&ms, b->tev[2 * k], b->tev[2 * k + 1]));
        t += ms;
    }
    float span = 0.f;
    BCK(cudaEventElapsedTime(&span, b->tev[0], b->tev[2 * (size_t)b->tev_used - 1]));
    *field_ms = t;
    *launches = b->tev_used;
    *span_ms = span;
    return GLASMA_OK;
}
extern "C" int32_t glasma_push_variants(void) { return push_variants(); }
extern "C" int32_t glasma_batch_push_variant(const glasma_batch* b) { return b ? b->pvar : GLASMA_ERR_INVALID; }
extern "C" glasma_status glasma_batch_set_push_variant(glasma_batch* b, int32_t v) {
    if (!b || !b->initialised) return bfail(GLASMA_ERR_INVALID, "batch not initialised");
    if (v < 0 || v >= push_variants()) return bfail(GLASMA_ERR_INVALID, "no such push variant");
    if (v == b->pvar) return GLASMA_OK;
    b->pvar = v;
    if (b->graph_ready) {
        cudaGraphExecDestroy(b->exec);
        b->graph_ready = false;
    }
    return GLASMA_OK;
}
// times the batched field kernel of every variant over the first `steps` iterations
// (from the initial state, one untimed warm-up iteration first) and keeps the fastest;
// then times every push kernel over `steps` iterations starting where the particles of
// every event are formed, and keeps the fastest
extern "C" glasma_status glasma_batch_tune(glasma_batch* b, int32_t steps, int32_t* chosen, double* ms) {
    if (!b || !b->initialised) return bfail(GLASMA_ERR_INVALID, "batch not initialised");
    if (steps < 1) return bfail(GLASMA_ERR_INVALID, "steps must be positive");
    const int nv = field_variants(b->prec);
    const int K = std::min<int>(steps + 1, b->max_iter);
    const size_t sa = step_args_size(b->prec), pa = push_args_size(b->prec);
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0));
    BCK(cudaEventCreate(&e1));
    int best = 0;
    double best_ms = 1e300;
    for (int v = 0; v < nv; v++) {
        glasma_status s = glasma_batch_set_variant(b, v);
        if (s != GLASMA_OK) return s;
        BCK(enqueue_restore(b));
        float t = 0;
        for (int k = 0; k < K; k++) {
            const int act = b->active[k];
            if (act == 0) break;
            if (k == 1) BCK(cudaEventRecord(e0, b->st));
            BCK(launch_field_step_variant(b->prec, v, (char*)b->step_args + (size_t)k * b->E * sa, b->gtiles_dev,
                                          b->gtiles_upto[act], b->st));
        }
        BCK(cudaEventRecord(e1, b->st));
        BCK(cudaEventSynchronize(e1));
        if (K > 1) BCK(cudaEventElapsedTime(&t, e0, e1));
        if (ms) ms[v] = t;
        if (t < best_ms) { best_ms = t; best = v; }
    }
    if (chosen) *chosen = best;
    glasma_status s = glasma_batch_set_variant(b, best);
    if (s != GLASMA_OK) return s;
    // push kernels: the window of `steps` iterations after the latest formation step
    int k0 = 0;
    for (const auto& x : b->ev) k0 = std::max(k0, x.n_form - 1);
    k0 = std::min(k0, std::max(0, b->max_iter - steps));
    const int k1 = std::min(b->max_iter, k0 + steps);
    int pbest = 0;
    double pbest_ms = 1e300;
    std::vector<cudaEvent_t> ev(2 * (size_t)std::max(1, k1 - k0));
    for (auto& x : ev) BCK(cudaEventCreate(&x));
    for (int v = 0; v < push_variants(); v++) {
        // each push kernel is timed with the field launches of its iterations: the record
        // push needs field launches that also write its records, and that cost is its own
        const bool rec = !b->any_sub && v == PUSH_VARIANT_RECORD;
        BCK(enqueue_restore(b));
        for (int k = 0; k < k1; k++) {
            const int act = b->active[k];
            if (act == 0) break;
            if (k >= k0) BCK(cudaEventRecord(ev[2 * (k - k0)], b->st));
            BCK(launch_field_step_variant(b->prec, b->fvar, (char*)b->step_args + (size_t)k * b->E * sa,
                                          b->gtiles_dev, b->gtiles_upto[act], b->st, rec));
            BCK(launch_push_batched(b->prec, b->any_sub ? PUSH_VARIANT_SUB : v, (char*)b->push_args + (size_t)k * b->E * pa, b->pitems_dev,
                                    b->pitems_upto[act], b->st));
            if (k >= k0) BCK(cudaEventRecord(ev[2 * (k - k0) + 1], b->st));
        }
        BCK(cudaStreamSynchronize(b->st));
        double t = 0;
        for (int k = k0; k < k1 && b->active[k]; k++) {
            float a = 0;
            BCK(cudaEventElapsedTime(&a, ev[2 * (k - k0)], ev[2 * (k - k0) + 1]));
            t += a;
        }
        if (t < pbest_ms) { pbest_ms = t; pbest = v; }
    }
    for (auto& x : ev) cudaEventDestroy(x);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return glasma_batch_set_push_variant(b, pbest);
}

// particles of event i after a run, original order (host arrays of n_particles; NULL skips)
extern "C" glasma_status glasma_batch_get_particles(glasma_batch* b, int32_t event, double* x, double* y, double* eta,
                                                    double* px, double* py, double* peta, double* Q) {
    if (!b || event < 0 || event >= b->E) return bfail(GLASMA_ERR_INVALID, "bad arguments");
    const BatchEvent& e = b->ev[b->pos[event]];
    const size_t np = e.np;
    if (np == 0) return GLASMA_OK;
    double* stage = (double*)b->scratch;  // 14 np doubles; the scratch holds >= 2 n_max^2 * 8 * 16 bytes
    if (14 * np * 8 > ic_scratch_bytes(b->nmax, b->fft_work)) return bfail(GLASMA_ERR_NOSPACE, "scratch too small");
    BCK(launch_part_to_canonical(b->prec, e.P, e.np, e.n, stage, b->st));
    std::vector<double> h(14 * np);
    BCK(cudaMemcpyAsync(h.data(), stage, 14 * np * 8, cudaMemcpyDeviceToHost, b->st));
    BCK(cudaStreamSynchronize(b->st));
    double* outs[6] = {x, y, eta, px, py, peta};
    for (int k = 0; k < 6; k++)
        if (outs[k]) memcpy(outs[k], h.data() + k * np, np * 8);
    if (Q)
        for (size_t j = 0; j < np; j++)
            for (int a = 0; a < 8; a++) Q[8 * j + a] = h[(6 + a) * np + j];
    return GLASMA_OK;
}

extern "C" int64_t glasma_batch_launches(const glasma_batch* b, int32_t mode) {
    if (!b || !b->initialised) return GLASMA_ERR_INVALID;
    int64_t L = 0;
    if (mode == GLASMA_BATCH_PER_EVENT) {
        for (const auto& x : b->ev) L += (x.n_steps - 1) + std::max(0, x.n_steps - x.n_form) * (x.np > 0);
    } else if (mode == GLASMA_BATCH_PERSISTENT) {
        L = 1;
    } else {
        for (int k = 0; k < b->max_iter; k++) L += b->active[k] ? 2 : 0;
    }
    return L;
}

extern "C" void glasma_batch_destroy(glasma_batch* b) {
    if (!b) return;
    if (b->graph_ready) cudaGraphExecDestroy(b->exec);
    for (auto& e : b->tev)
        if (e) cudaEventDestroy(e);
    for (auto& e : b->sev)
        if (e) cudaEventDestroy(e);
    if (b->st2) cudaStreamDestroy(b->st2);
    batch_free_persistent(b);
    delete b;
}
