/*
 * glasma.h - C ABI of the GB300 (sm_103a) library for the data-parallel hot path
 * of arXiv:2307.07999 (Avramescu, Baran, Greco, Ipp, Mueller, Ruggieri, "Heavy
 * quark kappa and jet qhat transport coefficients in the Glasma early stage of
 * heavy-ion collisions"):
 *
 *   - boost-invariant SU(3) Glasma fields on the transverse lattice, evolved by a
 *     leapfrog of gauge links and chromo-electric fields built from plaquettes
 *     and staples (Sec. 1, "Glasma", Eq. 1);
 *   - test particles under Wong's equations with the colored particle-in-cell
 *     method: each push gathers E and B at the particle's cell, advances x and p
 *     and rotates the color charge Q with the links it crosses (Sec. 1,
 *     "Probes in Glasma", Eq. 2);
 *   - the momentum broadening <dp_i^2>(tau) = <p_i^2(tau) - p_i^2(tau_form)>
 *     from which kappa and qhat follow by d/dtau (Sec. 2, Eq. 3).
 *
 * Units: physical inputs in GeV and fm; internally lattice units (a = 1, the
 * coupling g absorbed into the fields).  Outputs of broadening_accumulate are
 * in GeV^2 with tau in fm/c.
 *
 * Memory: the library never allocates device memory for field or particle
 * state.  The caller passes one device workspace per context (size from the
 * matching *_workspace_bytes call), 256-byte aligned, owned by the caller and
 * kept alive until the context is destroyed.  Host buffers passed to the calls
 * are caller-owned and only read or written during the call.
 *
 * Streams: every call is ordered on the CUDA stream given at creation (NULL =
 * legacy default stream).  Calls that return data to the host synchronise that
 * stream; the others only enqueue work.
 *
 * Errors: every call returns a glasma_status; no C++ exception crosses the ABI.
 * glasma_last_error() returns a thread-local message for the last failure.
 * A context whose call failed with GLASMA_ERR_CUDA should be destroyed.
 */
#ifndef GLASMA_H
#define GLASMA_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GLASMA_OK = 0,
    GLASMA_ERR_INVALID = -1,   /* bad argument, size or call order */
    GLASMA_ERR_CUDA = -2,      /* a CUDA or cuFFT call failed */
    GLASMA_ERR_NONFINITE = -3, /* a monitor found NaN/Inf */
    GLASMA_ERR_TIMEOUT = -4,   /* a bounded device wait ran out */
    GLASMA_ERR_NOCONV = -5,    /* the tau = 0+ link solve left links unconverged */
    GLASMA_ERR_NOSPACE = -6    /* the workspace is smaller than required */
} glasma_status;

typedef enum { GLASMA_FP64 = 0, GLASMA_FP32 = 1 } glasma_precision;

/* Glasma event (Sec. 1, "Glasma": MV model, the saturation-type scale g^2 mu is
 * the only physical parameter besides the lattice). */
typedef struct {
    int32_t n;               /* transverse lattice sites per side (periodic n x n) */
    int32_t n_sheets;        /* longitudinal color sheets of the MV charges */
    double L_fm;             /* transverse box size; lattice spacing a = L / n */
    double g2mu_GeV;         /* MV charge scale g^2 mu */
    double m_ir_GeV;         /* infrared regulator of the Poisson solve */
    double dtau_over_a;      /* leapfrog step in units of a (1/8) */
    double tau_end_fm;       /* evolution end; n_steps = ceil(tau_end / dtau) */
    int32_t precision;       /* glasma_precision of the evolution */
    int32_t reunit_every;    /* FP64 Gram-Schmidt of the links every k steps (0: never) */
    int32_t expanding;       /* 1: boost-invariant Milne evolution; 0: static box (tests) */
    int32_t newton_max_iter; /* tau = 0+ link solve: iteration cap per attempt */
    double newton_tol;       /* tau = 0+ link solve: residual ||r||_2 target */
    uint64_t seed;           /* Philox key of the MV charges */
} glasma_params;

/* Test-particle ensemble (Sec. 2, toy-model initialisation: uniform in the
 * transverse plane, eta = 0, fixed initial momentum, formed at tau_form). */
typedef struct {
    int32_t n_particles;
    int32_t init_kind;       /* 0: |p_T| uniform in [p_min, p_max], isotropic azimuth;
                                1: along +x with |p| uniform in [p_min, p_max] */
    double mass_GeV;         /* 0 allowed (massless partons) */
    double tau_form_fm;      /* activation step = round(tau_form / dtau) */
    double p_min_GeV, p_max_GeV;
    double q2, q3;           /* Casimirs of Q (4 and 10/3 for <QQ> = 1/2, <QQQ> = d/4) */
    int32_t bin_every;       /* counting sort of the particles by cell every k steps (0: never) */
    int32_t integrator;      /* momentum kick of Eq. 2: 0 explicit first order (magnetic term with the
                                pre-step momentum); 1 Boris (half electric kick, norm-preserving
                                rotation about Q.B, half electric kick; the Christoffel decay of
                                p_eta^ applied exactly over each half step): second order */
    int32_t substeps;        /* particle steps per field step (0 or 1: one).  s > 1: s steps of dtau/s,
                                each gathering the fields of the field step at the particle's
                                current cell (at most 64; a batch with such events pushes them
                                with a kernel of its own, not the tuned variants, and rejects
                                GLASMA_BATCH_PERSISTENT) */
    int32_t interp;          /* field gather: 0 nearest grid point (the site at the lower-left corner of
                                the particle's cell); 1 cloud in cell (the four sites around the
                                particle, their fields carried to that site by the links, x before
                                y, bilinear weights; batches as for substeps > 1) */
    uint64_t seed;           /* Philox key of positions, momenta and Haar rotations */
} cpic_params;

/* Lattice-correlator estimators (Sec. 2, "Lattice correlators", Eqs. 4 and 5). */
typedef struct {
    double tau_start_fm;     /* first step = round(tau_start / dtau) (as for particles formed then), >= 1 */
    double ox0;              /* offset of the lightlike paths in their start cells, [0, 1) */
} corr_params;

typedef struct glasma_ctx glasma_ctx;
typedef struct cpic_ctx cpic_ctx;
typedef struct glasma_corr glasma_corr;
typedef struct glasma_batch glasma_batch;
typedef struct glasma_mlp glasma_mlp;

/* ------------------------------------------------------------------ fields */

/* Device workspace needed by glasma_create for these parameters (bytes), or a
 * negative glasma_status if the parameters are invalid. */
int64_t glasma_workspace_bytes(const glasma_params* p);

/* Creates a field context on the current CUDA device.  workspace: device
 * pointer (>= glasma_workspace_bytes(p) bytes, 256-byte aligned); stream: a
 * cudaStream_t or NULL.  The state is undefined until glasma_init or
 * glasma_init_from_host. */
glasma_status glasma_create(const glasma_params* p, void* workspace, int64_t workspace_bytes,
                            void* stream, glasma_ctx** out);

/* MV initial conditions on the device (Sec. 1, Eq. 1 and the tau = 0+ matching),
 * leaving the state at step 1 (U, phi at tau = dtau; E = 0, pi = pi(0) at dtau/2).
 * Returns GLASMA_ERR_NOCONV if some links did not reach newton_tol (the state
 * is still usable; glasma_ic_stats reports how many). Synchronises. */
glasma_status glasma_init(glasma_ctx* g);

/* Newton statistics of the last glasma_init: failures, mean and max iterations. */
glasma_status glasma_ic_stats(const glasma_ctx* g, int64_t* failures, double* mean_iter,
                              int32_t* max_iter);

/* Loads a state from host memory in the canonical layout, site s = x + n*y:
 *   U   double[n*n][2][3][3][2]  (links U_x, U_y, complex row-major, re/im)
 *   E   double[n*n][2][8]        (E_x^a, E_y^a at tau_{step-1/2})
 *   phi double[n*n][8], pi double[n*n][8]
 * step: the leapfrog index of the state (U, phi at tau = step*dtau). Synchronises. */
glasma_status glasma_init_from_host(glasma_ctx* g, const double* U, const double* E,
                                    const double* phi, const double* pi, int32_t step);

/* Copies the current state to host memory in the canonical layout (any pointer
 * may be NULL to skip that field) and returns its step. Synchronises. */
glasma_status glasma_get_state(glasma_ctx* g, double* U, double* E, double* phi, double* pi,
                               int32_t* step);

/* Advances the fields by n_steps leapfrog steps (Sec. 1, "Glasma": the boost-invariant
 * Yang-Mills equations on the transverse lattice of gauge links and plaquettes; kick of
 * E_i and pi at tau_n by minus the group derivative of the lattice potential, built from
 * the plaquettes, their staples and the covariant differences of phi; drift of U_i and
 * phi with tau_{n+1/2}).  Enqueue only.  GLASMA_ERR_INVALID before an initial state
 * (or at tau = 0 in the expanding evolution); a failed launch, GLASMA_ERR_CUDA. */
glasma_status glasma_step(glasma_ctx* g, int32_t n_steps);

/* FP64 monitors of the current state (synchronises):
 *   out[0] Gauss-law violation relative to the scale of its terms
 *   out[1..4] eps_E,T, eps_B,T, eps_E,L, eps_B,L (lattice units, E and pi at tau_{n-1/2})
 *   out[5] max link unitarity deviation, out[6] tau (lattice units), out[7] nonfinite count */
glasma_status glasma_diagnostics(glasma_ctx* g, double out[8]);

void glasma_destroy(glasma_ctx* g);

/* The monitors of glasma_diagnostics for callers that cannot allocate device
 * memory (code handed only the buffers it reads, e.g. a plugin or host callback
 * inside another framework, or a process whose device memory pool is fully
 * reserved): no context, no workspace.  The paper has no counterpart; this is
 * a deployment aid.
 *   fields: device pointer to one field buffer in the library's plane layout
 *           (56 state planes of n*n reals of the given precision, site s = x + n*y:
 *           U_x rows 0-1 as 12 planes (entry-major, re then im), U_y likewise,
 *           E_x^a, E_y^a, phi^a, pi^a as 8 planes each; the planes are grouped
 *           by eight, interleaved per site: plane p of site s is element
 *           ((p / 8) * n*n + s) * 8 + p % 8), read only, 16-byte aligned.  The
 *           library's own buffers carry an eighth group (planes 56-63: the
 *           plaquettes a field step leaves for the push), which is not read here.
 *   tau: tau in lattice units (divides E and D phi in the expanding case).
 *   out: host double[8], as glasma_diagnostics.
 *   expanding: 1 the Milne evolution (tau > 0 required), 0 the static box.
 * Scratch: a file-scope device array of 4096 x 8 doubles (256 KB) that every
 * GPU which loads the library holds until the process exits; n*n above
 * 1,048,576 sites, or an unaligned buffer, is rejected with GLASMA_ERR_INVALID, and so is
 * a buffer that is not device (or managed) memory of the current device.  Each call
 * looks up the array's address on the current device (cudaGetSymbolAddress, which
 * allocates nothing), so it stays right across a device reset.  All calls share the
 * array: calls that overlap on the GPU (other streams or threads) race.  Allocates
 * nothing.  Synchronous: it copies the result to the host and waits for the stream, so
 * it cannot be captured (a capturing stream is refused with GLASMA_ERR_INVALID).
 * Non-finite values: GLASMA_ERR_NONFINITE with out filled. */
glasma_status glasma_diagnostics_noalloc(const void* fields, int32_t n, int32_t precision,
                                         int32_t expanding, double tau, void* stream, double out[8]);

/* ------------------------------------------------------------------ particles */

int64_t cpic_workspace_bytes(const glasma_params* gp, const cpic_params* p);

/* Creates a particle ensemble bound to the field context g (which must outlive it). */
glasma_status cpic_create(glasma_ctx* g, const cpic_params* p, void* workspace,
                          int64_t workspace_bytes, cpic_ctx** out);

/* Philox initial state (Sec. 1: Q0 in the Cartan subalgebra with the given
 * Casimirs, Q = U Q0 U^dag with Haar U; Sec. 2: toy-model positions and momenta). */
glasma_status cpic_init(cpic_ctx* c);

/* Loads particle states from host (double[n_particles] each; Q double[n][8]; p0
 * double[n][3] = lab momentum at formation; x, y continuous in [0, n)). */
glasma_status cpic_init_from_host(cpic_ctx* c, const double* x, const double* y,
                                  const double* eta, const double* px, const double* py,
                                  const double* peta, const double* Q, const double* p0);

/* Copies particle states to host in the original particle order (NULL skips). */
glasma_status cpic_get_particles(cpic_ctx* c, double* x, double* y, double* eta, double* px,
                                 double* py, double* peta, double* Q);

/* Coupled step (Sec. 1, "Probes in Glasma", Eq. 2: Wong's equations solved by the
 * colored particle-in-cell method): n_steps x (field step as glasma_step; then, if
 * tau_n >= tau_form, push every particle: gather E and B at its nearest-grid-point cell
 * from the fields of tau_n, kick p by the color Lorentz force Q.(E + v x B) in Milne
 * coordinates, drift x, y, eta, and rotate Q by exp(-i phi deta) and by the link of every
 * cell face it crosses; then add its broadening terms to the row of tau_{n+1}).
 * Enqueue only; GLASMA_ERR_INVALID on a negative count or an uninitialised context. */
glasma_status cpic_push(cpic_ctx* c, int32_t n_steps);

/* Coupled step for several ensembles in the same event (Sec. 2: charm and beauty quarks,
 * or jets of several momenta, probing one Glasma): n_steps x (one field step; then the
 * push of every ensemble, each as in cpic_push; then the sorts that are due).  The
 * ensembles with one particle step per field step and the nearest-grid-point gather are
 * pushed together, up to eight per launch, their 128-particle blocks interleaved so that
 * ensembles sorted by cell read the same field lines once; the others are pushed alone.
 * Each ensemble's particles come out exactly as when it is pushed alone (its table up to
 * the order of the FP64 block sums).  cs: host array of n_ctx >= 1 distinct ensembles, all
 * created on the same field context; each ensemble keeps its own mass, formation step,
 * integrator and broadening table.  A bad list is rejected with GLASMA_ERR_INVALID before
 * any work is enqueued.  Enqueue only. */
glasma_status cpic_push_many(cpic_ctx* const* cs, int32_t n_ctx, int32_t n_steps);

/* Broadening table (Sec. 2, "Quantifying the effect of Glasma": dp_i^2(tau) =
 * p_i^2(tau) - p_i^2(tau_form), averaged over the particles; the FP64 sums are
 * accumulated on the GPU at every push).  Synchronises.  Rows r = 0..n-1 from the first
 * pushed step (tau_form, or the field step at particle initialisation if later) to the
 * current step, each {tau_fm, <dp_x^2>, <dp_y^2>, <dp_z^2> (GeV^2), particle count},
 * p_z the lab longitudinal momentum.  host_out: caller-owned double[cap_rows][5];
 * GLASMA_ERR_NOSPACE if cap_rows is too small (nothing useful written). */
glasma_status broadening_accumulate(cpic_ctx* c, double* host_out, int64_t cap_rows,
                                    int64_t* n_rows);

/* Transport coefficients of Eq. 3 (Sec. 2): kappa_i = d<dp_i^2>/dtau for heavy quarks,
 * with i = L (the beam axis z) and T (x + y); qhat_i for jets along x, with i = z, y.  Also
 * the paragraph's anisotropy, <dp_L^2>/<dp_T^2> (heavy quarks) or <dp_z^2>/<dp_y^2> (jets).
 * The derivative is taken on the table's own tau grid: (f[r+1] - f[r-1])/(tau[r+1] -
 * tau[r-1]) inside, the one-sided secant at the first and last rows (0 for a one-row
 * table); "total" is the sum of the transverse and longitudinal coefficients.
 *   table: host double[rows][stride], stride >= 4, rows {tau, <dp_x^2>, <dp_y^2>, <dp_z^2>,
 *          ...} with tau strictly increasing (broadening_accumulate and
 *          glasma_batch_broadening write stride 5; any pooled table of that form works);
 *   kind:  GLASMA_HEAVY_QUARKS or GLASMA_JETS_X;
 *   out:   host double[rows][8] = {tau, d<dp_x^2>/dtau, d<dp_y^2>/dtau, d<dp_z^2>/dtau,
 *          transverse, longitudinal, total, anisotropy} (units of the table per unit of
 *          its tau: GeV^2/fm for the tables above; the anisotropy is NaN where the
 *          transverse broadening is zero, e.g. at the formation row).
 * Host computation in FP64, no device work; GLASMA_ERR_INVALID on a null pointer, a bad
 * kind or stride, or a tau column that does not increase. */
enum { GLASMA_HEAVY_QUARKS = 0, GLASMA_JETS_X = 1 };
glasma_status broadening_transport(const double* table, int64_t rows, int32_t stride, int32_t kind,
                                   double* out);

/* Checkpoint and resume of a coupled run (the paper has no counterpart: a long evolution,
 * e.g. 820 steps of 1024^2 with millions of partons, can be stopped and continued with
 * identical results).  A blob is a small header followed by the raw device image:
 *   field context: the current field buffer and its step (attached correlator
 *     estimators are not included);
 *   particle ensemble: the particle planes (original order kept), the FP64 broadening
 *     sums of every row, the formation step and the sorting counter.
 * *_state_bytes: the blob size for this context (negative glasma_status on a null
 * context).  export: host must hold that many bytes; synchronises.  import: into a
 * context created with the same parameters (precision, lattice, dtau, tau_end,
 * expanding; for particles also count, mass and integrator), otherwise
 * GLASMA_ERR_INVALID and nothing is changed; synchronises.  A run continued from the
 * blobs repeats the original bit for bit (the broadening sums to the order of their
 * FP64 atomic additions). */
int64_t glasma_state_bytes(const glasma_ctx* g);
glasma_status glasma_export_state(glasma_ctx* g, void* host, int64_t bytes);
glasma_status glasma_import_state(glasma_ctx* g, const void* host, int64_t bytes);
int64_t cpic_state_bytes(const cpic_ctx* c);
glasma_status cpic_export_state(cpic_ctx* c, void* host, int64_t bytes);
glasma_status cpic_import_state(cpic_ctx* c, const void* host, int64_t bytes);

/* Maximum drift of the Casimirs q2, q3 over all particles (synchronises). */
glasma_status cpic_casimir_drift(cpic_ctx* c, double out[2]);

void cpic_destroy(cpic_ctx* c);

/* ------------------------------------------------------------------ lattice correlators
 * The momentum broadening of static quarks (m -> infinity, Eq. 4) and of lightlike jets
 * along +x (p_x -> infinity, Eq. 5) from the Glasma fields alone, for every site:
 *   static:    I_i(x) = sum over steps of dtau E_i(x),  <dp_i^2> = <Tr I_i^2>_x
 *   lightlike: the path from x0 moves one lattice unit of x per unit of tau from offset
 *              ox0; J_i(x0) = sum of dtau W F_i W^dag with F = (E_x, E_y - B_z, E_z + B_y)
 *              at the path's cell and W the product of the x-links the path crossed;
 *              <dp_i^2> = <Tr J_i^2>_x0
 * with the site-centred fields of the particle push (time-centred E_x, E_y averaged over
 * the two links at the site, E_z = pi, clover B_z, covariant differences of phi).  These
 * are the Q-averaged limits of the Wong push (a charge Q parallel transported along the
 * path collects Q.J).  The estimator attaches to a field context and advances with every
 * field step of glasma_step and cpic_push from its first step; one per context.
 * Workspace: caller-owned device memory, 256-byte aligned (66 reals per site in the
 * context's precision, plus FP64 sums).  Destroy it before its context. */
int64_t corr_workspace_bytes(const glasma_params* p);
glasma_status corr_create(glasma_ctx* g, const corr_params* p, void* workspace, int64_t workspace_bytes,
                          glasma_corr** out);
/* host_out [rows][7] = {tau_fm, static <dp_x^2>, <dp_y^2>, <dp_z^2>, lightlike <dp_x^2>,
 * <dp_y^2>, <dp_z^2>} in GeV^2, FP64, from the first step (zeros) to the current one.
 * Synchronises. */
glasma_status corr_table(glasma_corr* c, double* host_out, int64_t cap, int64_t* n_rows);
void corr_destroy(glasma_corr* c);

/* ------------------------------------------------------------------ learned warm start
 * A 36 -> 128 -> 128 -> 16 tanh network (BF16 weights, FP32 accumulation) that
 * corrects, for each link, the starting point of the tau = 0+ Newton solve:
 *   U0 = exp(i (d_s + d_net).t) U1 U2,
 *   d_s = -c/2 - (3/8) i[a1, c] - (1/8) i[a2, c],  a_k = 2 Im Tr[t^a U_k], c = i[a1, a2]
 * (d_s: the solution's offset from U1 U2 through third order in the link fields).
 * The Newton iteration still decides every link to newton_tol.  The paper has no
 * learned component; this only shortens the initial-condition solve.
 * Inputs (36): a1, a2, c, d_s + c/2, |a1|^2, |a2|^2, a1.a2, |c|^2;
 * targets (8): d - d_s with d^a = 2 Im Tr[t^a U (U1 U2)^dag] of the Newton solution U. */

int64_t glasma_mlp_workspace_bytes(void);
/* Glorot-initialised network in a caller-owned device workspace (256-byte aligned). */
glasma_status glasma_mlp_create(void* workspace, int64_t workspace_bytes, uint64_t seed, void* stream,
                                glasma_mlp** out);
void glasma_mlp_destroy(glasma_mlp* m);
/* Fixed input / target scalings: set them, or fit them to the RMS of a data set
 * (device float arrays X[N][36], T[N][8]). */
glasma_status glasma_mlp_set_scales(glasma_mlp* m, float x_scale, float y_scale);
glasma_status glasma_mlp_fit_scales(glasma_mlp* m, const float* X, const float* T, int64_t N);
/* Mini-batch Adam (FP32 master weights) over N pairs for some epochs, batches in
 * the given order; last_loss: mean loss of the last epoch. Synchronises. */
glasma_status glasma_mlp_train(glasma_mlp* m, const float* X, const float* T, int64_t N, int32_t epochs,
                               int32_t batch, float lr, double* last_loss);
/* Loss and FP32 gradients of one batch without updating (grads_host: float[23312]
 * in the order W1[128][36], b1[128], W2[128][128], b2[128], W3[16][128], b3[16],
 * or NULL). Synchronises. */
glasma_status glasma_mlp_loss_grad(glasma_mlp* m, const float* X, const float* T, int64_t N, double* loss,
                                   float* grads_host);
/* Predicted correction d_net (device float Y[N][8]) for device features X[N][36];
 * enqueue only. */
glasma_status glasma_mlp_predict(glasma_mlp* m, const float* X, int64_t N, float* Y);
/* FP32 master parameters (host float[23312], same order) and scalings (float[2], or NULL). */
glasma_status glasma_mlp_get_params(glasma_mlp* m, float* host, float* scales);
glasma_status glasma_mlp_set_params(glasma_mlp* m, const float* host);
/* Features X[2 n*n][36] and targets T[2 n*n][8] (device float, link l = 2 s + d) of the
 * last glasma_init / glasma_init_warm of the context. Synchronises. */
glasma_status glasma_ic_dataset(glasma_ctx* g, float* X, float* T);
/* As glasma_init, every link's Newton solve starting from U0 above (then from
 * U1 U2, then from 1 if an attempt stalls). Synchronises. */
glasma_status glasma_init_warm(glasma_ctx* g, glasma_mlp* m);

/* ------------------------------------------------------------------ event batches
 * Many events of uneven lattice sizes, each with its own particle ensemble,
 * advanced together; <dp_i^2> averages over particles and events (Sec. 2). */

typedef enum {
    GLASMA_BATCH_GRAPH = 0,      /* per step: one field launch over all active events' tiles and one push
                                    launch over their particles; the whole run is one CUDA graph */
    GLASMA_BATCH_PERSISTENT = 1, /* one persistent cooperative kernel for the whole run: field and push
                                    phases separated by a bounded grid barrier */
    GLASMA_BATCH_PER_EVENT = 2,  /* plain loop: one event after the other, one launch per kernel */
    GLASMA_BATCH_EAGER = 3       /* the launches of GLASMA_BATCH_GRAPH issued without a graph */
    /* (mode 4, a field step fused with the push of each tile's particles after binning them by
       tile, was measured 4-5x slower than GLASMA_BATCH_GRAPH and is no longer offered) */
} glasma_batch_mode;

/* Workspace for n_events events: ev[i], pp[i] give event i (all with the same
 * precision and expanding = 1). */
int64_t glasma_batch_workspace_bytes(const glasma_params* ev, const cpic_params* pp, int32_t n_events);
glasma_status glasma_batch_create(const glasma_params* ev, const cpic_params* pp, int32_t n_events,
                                  void* workspace, int64_t workspace_bytes, void* stream,
                                  glasma_batch** out);
/* MV initial conditions and particles of every event (kept as the restart
 * state of each run); ic_failures: unconverged tau = 0+ links. Synchronises. */
glasma_status glasma_batch_init(glasma_batch* b, int64_t* ic_failures);
/* One run: every event from its initial state to its own tau_end (enqueue only).
 * GLASMA_BATCH_GRAPH needs a created stream (not NULL / the legacy default stream). */
glasma_status glasma_batch_run(glasma_batch* b, int32_t mode);
/* Site-updates and particle-steps of one run. */
glasma_status glasma_batch_work(const glasma_batch* b, int64_t* site_updates, int64_t* particle_steps);
/* Broadening table of event i after a run (rows as in broadening_accumulate). */
glasma_status glasma_batch_broadening(glasma_batch* b, int32_t event, double* host_out, int64_t cap_rows,
                                      int64_t* n_rows);
/* Monitors of event i's final state (as glasma_diagnostics). */
glasma_status glasma_batch_diagnostics(glasma_batch* b, int32_t event, double out[8]);
/* Raw initial state of all events (device layout, event order): size, copy out,
 * copy in (the next glasma_batch_run starts from it).  A checkpoint of the
 * batch's starting point; export synchronises, import only enqueues.  The import
 * source may be host memory or device memory: a caller that streams inputs can copy
 * the next state from pinned host memory into a device staging buffer of its own on
 * another stream while the current run executes, then import from that buffer (a
 * device-to-device copy on the batch stream, ordered after the caller's copy by the
 * caller, e.g. with an event). */
int64_t glasma_batch_state_bytes(const glasma_batch* b);
glasma_status glasma_batch_export_state(glasma_batch* b, void* host, int64_t bytes);
glasma_status glasma_batch_import_state(glasma_batch* b, const void* host, int64_t bytes);
/* One run of the graph mode's launches issued eagerly with CUDA events around every launch
 * (batch stream): main = the batched field kernel, other = the batched push (mode is
 * ignored).  Returns the total main-kernel time (ms), its launches, the site-updates it
 * performed, 0 particle-steps (the push is separate), and the total time of the pushes.
 * Synchronises. */
glasma_status glasma_batch_profile(glasma_batch* b, int32_t mode, double* main_ms, int64_t* main_launches,
                                   int64_t* main_sites, int64_t* main_particle_steps, double* other_ms);
/* Pushes on a second stream (graph and eager modes), with separate != 0: the push of
 * iteration k waits for field launch k, field launch k+2 for push k (the buffer it writes
 * is the one push k reads), so a push overlaps the next field launch; the run still ends
 * on the batch stream.  Results are unchanged.  The graph is captured again when this
 * changes. */
glasma_status glasma_batch_set_push_stream(glasma_batch* b, int32_t separate);
/* Kernel timing inside the timed runs themselves: with on != 0, the batched path (graph and
 * eager modes) brackets every batched field launch with CUDA event records, captured in
 * the graph as event-record nodes (the graph is captured again when this changes).
 * glasma_batch_graph_times then returns, for the last run, the summed duration of its
 * field launches (ms), their number, and the span from the first field launch's start to
 * the last one's end (ms).  Synchronises on the last event.  No counterpart in the paper:
 * measurement. */
glasma_status glasma_batch_set_graph_timing(glasma_batch* b, int32_t on);
glasma_status glasma_batch_graph_times(glasma_batch* b, double* field_ms, int64_t* launches, double* span_ms);
/* Bound of the GLASMA_BATCH_PERSISTENT mode's grid-barrier wait, in polls of about 100 ns
 * (0: the default 2^24, about 2 s; at most 2^40).  A CTA whose wait runs out raises the
 * kernel's error word and returns; every other CTA returns at its next barrier (each wait
 * is bounded the same way), so the launch always ends.  The next glasma_batch_broadening
 * of the batch then reports GLASMA_ERR_TIMEOUT once (the word is cleared when read), and
 * the next run starts from the initial state as usual.  Failure detection: a limit far
 * below a step's duration makes the wait run out on purpose.  Host only, no device work;
 * GLASMA_ERR_INVALID on a null batch or a limit out of range. */
glasma_status glasma_batch_set_wait_limit(glasma_batch* b, int64_t polls);
/* Particles of event i (original order; double[n] each, Q double[n][8]; NULL skips). */
glasma_status glasma_batch_get_particles(glasma_batch* b, int32_t event, double* x, double* y, double* eta,
                                         double* px, double* py, double* peta, double* Q);
/* Kernel launches of one run in the given mode. */
int64_t glasma_batch_launches(const glasma_batch* b, int32_t mode);
/* Tile shapes of the batched field step (graph and eager modes).  The FP32 kernel is
 * compiled for several (TX, TY, minimum resident CTAs per SM); FP64 has one.  The
 * per-site arithmetic is the same in every shape, so results do not depend on it.
 * glasma_batch_tune times each variant's field kernel over the first `steps`
 * iterations of the batch (restored to its initial state; one untimed warm-up
 * iteration first), keeps the fastest and returns it in *chosen, the times (ms) in
 * ms[variants] unless NULL.  Changing the variant drops the captured graph of the
 * graph mode (it is captured again at the next run).  Synchronises. */
int32_t glasma_field_tile_variants(int32_t precision);
glasma_status glasma_field_tile_shape(int32_t precision, int32_t variant, int32_t* tx, int32_t* ty,
                                      int32_t* min_ctas);
int32_t glasma_batch_variant(const glasma_batch* b);
glasma_status glasma_batch_set_variant(glasma_batch* b, int32_t variant);
glasma_status glasma_batch_tune(glasma_batch* b, int32_t steps, int32_t* chosen, double* ms);
/* Batched push kernels (graph and eager modes): 0 reads the fields through L1 (128-thread
 * blocks), 1 stages each particle's fields in shared memory first (cp.async); both gather
 * the 35 field groups around the particle's cell.  2, the record push: the field launch of
 * each step also writes, for every cell a particle occupies (cells stamped by the previous
 * push; every cell at the particles' first step), the pieces of the site-centred fields it
 * computes anyway, and the push reads that one contiguous record; the pushes and field
 * launches then stay on one stream (glasma_batch_set_push_stream has no effect).  3, the
 * split push: a force kernel gathers the fields and stores the six Q-contracted forces of
 * each particle, a move kernel kicks, drifts and rotates from them.  Same physics (results
 * equal to rounding: FP64 runs agree with the oracle to 1e-10 in every variant).  Events
 * with sub-steps or the cloud-in-cell gather always use a push of their own.
 * glasma_batch_tune also times them, each with the field launches of its iterations, over
 * `steps` iterations after the particles of every event are formed, and keeps the fastest. */
int32_t glasma_push_variants(void);
int32_t glasma_batch_push_variant(const glasma_batch* b);
glasma_status glasma_batch_set_push_variant(glasma_batch* b, int32_t variant);
void glasma_batch_destroy(glasma_batch* b);

const char* glasma_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
