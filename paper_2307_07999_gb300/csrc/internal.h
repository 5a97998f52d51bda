// Host-side launchers shared by the translation units of the library (no
// device code here).  prec: 0 = FP64 evolution, 1 = FP32 evolution.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

struct glasma_mlp;  // the warm-start network (mlp.cu)

namespace glasma {

constexpr int N_FIELD_PLANES = 64;
constexpr int N_PART_REAL_PLANES = 17;  // ox oy eta p0x p0y p0z dpx dpy peta Q[8]

inline size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// ---------------- fields
struct StepHost {
    const void* src;
    void* dst;
    int n;
    double tb, tp, dtau, ue, pe;
    int reunit;
    void* plaq;       // the buffer receiving the plaquettes of src's links (src itself)
    void* rec;        // gather records written by the REC kernels (null otherwise)
    const int* occ;   // occupancy stamps they test
    int epoch;        // the step index: a cell whose stamp equals it gets a record
    int all_rec;      // 1: every cell gets a record (the particles' first step)
};
// leapfrog coefficients of step n (state at tau_n = n dtau)
StepHost step_coeffs(const void* src, void* dst, int n, int step, double dtau, int expanding, int reunit);
// link re-projection after the drift of step s: 1 the FP64 Gram-Schmidt (every reunit_every
// steps), 2 the FP32 first-order renormalisation (every RENORM_EVERY steps otherwise;
// FP32 only), 0 none
// (every 2 steps: the 64-event batch of 128^2-512^2 lattices runs 1.3 % faster, but on one
// 512^2 event with 200k quarks the FP32-vs-FP64 error of <dp^2> doubles to 1.5e-5 and
// kappa's rises to 2.2e-4)
constexpr int RENORM_EVERY = 1;
inline int reunit_code(int reunit_every, int s) {
    if (reunit_every > 0 && (s + 1) % reunit_every == 0) return 1;
    return (s + 1) % RENORM_EVERY == 0 ? 2 : 0;
}
cudaError_t launch_field_step(int prec, const StepHost& a, cudaStream_t st);
// batched: args[n_ev], items[n_items] (device arrays), one CTA per item
cudaError_t launch_field_step_batched(int prec, const void* args_dev, const void* items_dev, int n_items,
                                      cudaStream_t st, bool rec = false);
int field_tile_x(int prec);
int field_tile_y(int prec);
int field_variants(int prec);
void field_variant_shape(int prec, int v, int* tx, int* ty, int* minb);
cudaError_t prepare_field_variants(int prec);
cudaError_t prepare_push_staged();
cudaError_t launch_field_step_variant(int prec, int v, const void* args, const void* items, int n_items,
                                      cudaStream_t st, bool rec = false);
// bytes of one cell's gather record (REC_STRIDE groups of 8 reals)
size_t record_bytes(int prec);
size_t step_args_size(int prec);
void pack_step_args(int prec, const StepHost& a, void* out);

// canonical host layout <-> device planes
cudaError_t launch_state_from_canonical(int prec, const double* dU, const double* dE, const double* dphi,
                                        const double* dpi, void* buf, int n, cudaStream_t st);
cudaError_t launch_state_to_canonical(int prec, const void* buf, double* dU, double* dE, double* dphi,
                                      double* dpi, int n, cudaStream_t st);
// monitors into mon[0..7] (zeroed here)
cudaError_t launch_monitors(int prec, const void* buf, int n, double tau_e, double* mon, cudaStream_t st);

// ---------------- particles
struct PartHost {
    int* cell; int* pid;
    void* planes;  // N_PART_REAL_PLANES planes of np reals, plane stride pstride (elements)
    size_t pstride;
};
PartHost part_layout(void* base, int np, int prec);
size_t part_bytes(int np, int prec);
struct PushHost {
    const void* fo; const void* fn;
    int n, np;
    double dtau, te, ichr, teh, mass;
    int expanding;
    int boris;           // momentum kick: 0 explicit, 1 Boris
    int nsub;            // particle steps per field step
    double hsub, tau0;   // their length dtau / nsub, and tau_n
    int interp;          // gather: 0 nearest grid point, 1 cloud in cell
    double dec0, dec1;   // Boris: p_eta^ decay factors tau_n/tau_{n+1/2}, tau_{n+1/2}/tau_{n+1} (1: static box)
    double* acc;
    const void* rec;     // record push: the gather records of this step
    int* occ;            // record push: occupancy stamps, set to epoch_next at the new cells
    int epoch_next;
    void* frc;           // split push: 6 planes of np reals (particle plane stride) of contracted fields
};
// the step-dependent coefficients of the push from tau_n = step * dtau to tau_{n+1}
inline void push_coeffs(PushHost& a, int step, double dtau, int expanding, int integrator, int substeps,
                        int interp) {
    const double tn = step * dtau, th = (step + 0.5) * dtau, t1 = (step + 1.0) * dtau;
    a.dtau = dtau;
    a.expanding = expanding;
    a.te = expanding ? tn : 1.0;
    a.ichr = expanding ? 1.0 / tn : 0.0;
    a.teh = expanding ? th : 1.0;
    a.boris = integrator == 1;
    a.dec0 = expanding ? tn / th : 1.0;
    a.dec1 = expanding ? th / t1 : 1.0;
    a.nsub = substeps > 1 ? substeps : 1;
    a.hsub = dtau / a.nsub;
    a.tau0 = tn;
    a.interp = interp;
}
cudaError_t launch_push(int prec, const PushHost& a, const PartHost& P, cudaStream_t st);
// up to PUSH_PACK_MAX ensembles of one event (no sub-steps, nearest grid point) in one launch
constexpr int PUSH_PACK_MAX = 8;
cudaError_t launch_push_pack(int prec, const PushHost* a, const PartHost* const* P, int n, cudaStream_t st);
// batched push: args[n_ev] (acc == nullptr: event idle this step), items {ev, j0} of 256 particles
size_t push_args_size(int prec);
void pack_push_args(int prec, const PushHost& a, const PartHost& P, void* out);
int push_variants();
// the batched push of batches with sub-stepped or cloud-in-cell events (global source, any
// cell; not tuned)
constexpr int PUSH_VARIANT_SUB = 99;
// the record push (tuned variant 2): the field launches of the same run write gather records
constexpr int PUSH_VARIANT_RECORD = 2;
// the split push (tuned variant 3): a force kernel (gather, contracted fields stored per
// particle) and a move kernel
constexpr int PUSH_VARIANT_SPLIT = 3;
// lattice-correlator estimators (kernels_corr.cu): state = I [24][ns], J [24][ns], W [18][ns]
size_t corr_state_bytes(int prec, int n);
cudaError_t launch_corr_reset(int prec, void* state, int n, cudaStream_t st);
cudaError_t launch_corr_step(int prec, const void* fo, const void* fn, int n, double te, double dtau, void* state,
                             int k_now, int k_next, double* acc, cudaStream_t st);
cudaError_t launch_push_batched(int prec, int variant, const void* args_dev, const void* items_dev, int n_items,
                                cudaStream_t st);
struct PushItemH { int ev, j0; };
struct TileItemH { int ev, x0, y0; };
cudaError_t launch_sort(int prec, const PartHost& a, const PartHost& b, int np, int ncell, int* count,
                        int* start, int* totals, cudaStream_t st);
size_t sort_scratch_ints(int ncell);
cudaError_t launch_part_init(int prec, const PartHost& P, int np, int n, int kind, double pmin, double pmax,
                             double q2, double q3, uint64_t seed, double mass, cudaStream_t st);
cudaError_t launch_part_from_canonical(int prec, const PartHost& P, int np, int n, const double* d /*[11+8][np]*/,
                                       cudaStream_t st);
cudaError_t launch_part_to_canonical(int prec, const PartHost& P, int np, int n,
                                     double* d /*[6+8][np], original order*/, cudaStream_t st);
cudaError_t launch_casimir_drift(int prec, const PartHost& P, int np, double q2, double q3, double* out2,
                                 cudaStream_t st);

// ---------------- initial conditions (FP64 scratch)
struct ICScratch {
    double* V1; double* V2;   // [ns][18]
    double* fft;              // real [8][ns]: charges rho, then Lambda
    double* spec;             // complex [8][n][n/2 + 1]: their half spectrum
    double* U;                // [ns][2][18]
    double* pi0;              // [ns][8]
    int* iters;               // [2 ns]
    double* res;              // [2 ns]
    void* fft_work; size_t fft_work_bytes;
    float* X;                 // [2 ns][36] warm-start features
    float* D;                 // [2 ns][8]  predicted starting corrections
    double* ktab;             // [n] lattice momenta 4 sin^2(pi k / n)
    int* nwt;                 // Newton passes: attempt [2 ns], iterations in it [2 ns], two link lists [2][2 ns]
    int* ncnt;                // list lengths [2]
};
size_t ic_scratch_bytes(int n, size_t fft_work_bytes);
ICScratch ic_layout(void* base, int n, size_t fft_work_bytes);
// full MV pipeline; writes the state at step 1 into buf; fails/iters summary into host ints
// mlp (nullable): the warm-start network proposes each link's Newton start
int ic_run(int prec, int n, int n_sheets, double g2mua, double m_ir_a, uint64_t seed, double dtau, double tol,
           int max_iter, const ICScratch& s, void* buf, cudaStream_t st, long long* fails, double* mean_it,
           int* max_it, const char** err, ::glasma_mlp* mlp = nullptr);
size_t ic_fft_work_bytes(int n, const char** err);
cudaError_t launch_ic_features(const ICScratch& s, int n, float* X, float* T, cudaStream_t st);
cudaError_t mlp_predict_dev(::glasma_mlp* M, const float* X, int64_t N, float* Y, cudaStream_t st);

}  // namespace glasma
