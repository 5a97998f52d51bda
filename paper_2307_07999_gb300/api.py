"""Thin Python surface over the C ABI: same names, argument marshalling only.

Device workspaces come from PyTorch (torch.empty on the CUDA device) and the
CUDA stream is torch's current stream unless one is given.  All compute runs
in libglasma.so.
"""
import ctypes as C

import numpy as np
import torch

from ._lib import GLASMA_HEAVY_QUARKS, GLASMA_JETS_X, CorrParams, CpicParams, GlasmaParams, check, lib

HBARC = 0.1973269804  # GeV fm


def _stream_ptr(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _workspace(nbytes, device):
    # 256-byte aligned device buffer owned by the caller (PyTorch's caching allocator)
    t = torch.empty(int(nbytes) + 256, dtype=torch.uint8, device=device)
    off = (-t.data_ptr()) % 256
    return t, t.data_ptr() + off


def _dp(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# ------------------------------------------------------------------ C-named calls
def glasma_create(params, workspace_ptr, nbytes, stream=None):
    h = C.c_void_p()
    check(lib().glasma_create(C.byref(params), C.c_void_p(workspace_ptr), nbytes, _stream_ptr(stream), C.byref(h)))
    return h


def glasma_init(handle):
    return lib().glasma_init(handle)


def glasma_step(handle, n_steps):
    check(lib().glasma_step(handle, n_steps))


def cpic_create(ghandle, params, workspace_ptr, nbytes):
    h = C.c_void_p()
    check(lib().cpic_create(ghandle, C.byref(params), C.c_void_p(workspace_ptr), nbytes, C.byref(h)))
    return h


def cpic_init(handle):
    check(lib().cpic_init(handle))


def cpic_push(handle, n_steps):
    check(lib().cpic_push(handle, n_steps))


def cpic_push_many(handles, n_steps):
    arr = (C.c_void_p * len(handles))(*[h.value if isinstance(h, C.c_void_p) else h for h in handles])
    check(lib().cpic_push_many(arr, len(handles), n_steps))


def broadening_accumulate(handle, cap):
    out = np.zeros((cap, 5))
    n = C.c_int64()
    check(lib().broadening_accumulate(handle, _dp(out), cap, C.byref(n)))
    return out[: n.value]


# ------------------------------------------------------------------ owning wrappers
class Glasma:
    """A field context with its PyTorch-owned workspace."""

    def __init__(self, n, L_fm, g2mu_GeV=2.0, m_ir_GeV=0.2, n_sheets=10, dtau_over_a=0.125, tau_end_fm=1.0,
                 precision=0, reunit_every=0, expanding=1, seed=1, newton_max_iter=100, newton_tol=1e-12,
                 device="cuda", stream=None):
        self.params = GlasmaParams(n, n_sheets, L_fm, g2mu_GeV, m_ir_GeV, dtau_over_a, tau_end_fm, precision,
                                   reunit_every, expanding, newton_max_iter, newton_tol, seed)
        nb = lib().glasma_workspace_bytes(C.byref(self.params))
        check(0 if nb >= 0 else nb)
        self._ws, ptr = _workspace(nb, device)
        self.handle = glasma_create(self.params, ptr, nb, stream)
        self.n = n
        self.a_fm = L_fm / n
        self.dtau = dtau_over_a

    def init(self):
        """MV initial conditions on the device; returns (failures, mean_iter, max_iter)."""
        st = lib().glasma_init(self.handle)
        if st not in (0, -5):
            check(st)
        return self.ic_stats()

    def ic_stats(self):
        f, m, x = C.c_int64(), C.c_double(), C.c_int32()
        check(lib().glasma_ic_stats(self.handle, C.byref(f), C.byref(m), C.byref(x)))
        return f.value, m.value, x.value

    def set_state(self, U, E, phi, pi, step):
        U = np.ascontiguousarray(U, dtype=np.complex128)
        E, phi, pi = (np.ascontiguousarray(a, dtype=np.float64) for a in (E, phi, pi))
        check(lib().glasma_init_from_host(self.handle, _dp(U), _dp(E), _dp(phi), _dp(pi), step))

    def export_state(self):
        """Checkpoint blob of the current fields (numpy uint8)."""
        nb = lib().glasma_state_bytes(self.handle)
        check(0 if nb >= 0 else nb)
        blob = np.empty(nb, dtype=np.uint8)
        check(lib().glasma_export_state(self.handle, blob.ctypes.data_as(C.c_void_p), nb))
        return blob

    def import_state(self, blob):
        blob = np.ascontiguousarray(blob, dtype=np.uint8)
        check(lib().glasma_import_state(self.handle, blob.ctypes.data_as(C.c_void_p), blob.size))

    def get_state(self):
        ns = self.n * self.n
        U = np.zeros((ns, 2, 3, 3), dtype=np.complex128)
        E = np.zeros((ns, 2, 8))
        phi = np.zeros((ns, 8))
        pi = np.zeros((ns, 8))
        st = C.c_int32()
        check(lib().glasma_get_state(self.handle, _dp(U), _dp(E), _dp(phi), _dp(pi), C.byref(st)))
        return U, E, phi, pi, st.value

    def step(self, n_steps=1):
        glasma_step(self.handle, n_steps)

    def diagnostics(self):
        out = np.zeros(8)
        st = lib().glasma_diagnostics(self.handle, _dp(out))
        if st not in (0, -3):
            check(st)
        return out

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            lib().glasma_destroy(h)
            self.handle = None


class WarmStartNet:
    """The warm-start network of the tau = 0+ link solve (see include/glasma.h)."""

    N_PARAMS = 23312
    SHAPES = (("W1", (128, 36)), ("b1", (128,)), ("W2", (128, 128)), ("b2", (128,)), ("W3", (16, 128)),
              ("b3", (16,)))

    def __init__(self, seed=7, device="cuda", stream=None):
        nb = lib().glasma_mlp_workspace_bytes()
        self._ws, ptr = _workspace(nb, device)
        h = C.c_void_p()
        check(lib().glasma_mlp_create(C.c_void_p(ptr), nb, seed, _stream_ptr(stream), C.byref(h)))
        self.handle = h

    @staticmethod
    def _t(x):
        assert x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()
        return C.c_void_p(x.data_ptr())

    def fit_scales(self, X, T):
        check(lib().glasma_mlp_fit_scales(self.handle, self._t(X), self._t(T), X.shape[0]))

    def set_scales(self, xs, ys):
        check(lib().glasma_mlp_set_scales(self.handle, xs, ys))

    def train(self, X, T, epochs=1, batch=4096, lr=1e-3):
        loss = C.c_double()
        check(lib().glasma_mlp_train(self.handle, self._t(X), self._t(T), X.shape[0], epochs, batch, lr,
                                     C.byref(loss)))
        return loss.value

    def loss_grad(self, X, T):
        loss = C.c_double()
        g = np.zeros(self.N_PARAMS, dtype=np.float32)
        check(lib().glasma_mlp_loss_grad(self.handle, self._t(X), self._t(T), X.shape[0], C.byref(loss), _dp(g)))
        return loss.value, self.unflatten(g)

    def predict(self, X):
        Y = torch.empty((X.shape[0], 8), dtype=torch.float32, device=X.device)
        check(lib().glasma_mlp_predict(self.handle, self._t(X), X.shape[0], self._t(Y)))
        return Y

    def params(self):
        p = np.zeros(self.N_PARAMS, dtype=np.float32)
        sc = np.zeros(2, dtype=np.float32)
        check(lib().glasma_mlp_get_params(self.handle, _dp(p), _dp(sc)))
        return self.unflatten(p), sc

    def set_params(self, d):
        flat = np.concatenate([np.asarray(d[k], dtype=np.float32).reshape(-1) for k, _ in self.SHAPES])
        check(lib().glasma_mlp_set_params(self.handle, _dp(flat)))

    @classmethod
    def unflatten(cls, flat):
        out, o = {}, 0
        for k, s in cls.SHAPES:
            n = int(np.prod(s))
            out[k] = flat[o:o + n].reshape(s)
            o += n
        return out

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            lib().glasma_mlp_destroy(h)
            self.handle = None


def ic_dataset(glasma):
    """Features [2 n^2, 36] and targets [2 n^2, 8] (device FP32) of the context's last
    initial condition."""
    nl = 2 * glasma.n * glasma.n
    X = torch.empty((nl, 36), dtype=torch.float32, device="cuda")
    T = torch.empty((nl, 8), dtype=torch.float32, device="cuda")
    check(lib().glasma_ic_dataset(glasma.handle, C.c_void_p(X.data_ptr()), C.c_void_p(T.data_ptr())))
    return X, T


def init_warm(glasma, net):
    """glasma_init_warm: MV initial conditions with the network's Newton starts."""
    st = lib().glasma_init_warm(glasma.handle, net.handle)
    if st not in (0, -5):
        check(st)
    return glasma.ic_stats()


class Correlators:
    """Lattice-correlator estimators (static quarks, Eq. 4; lightlike jets along +x,
    Eq. 5) attached to a Glasma context: they advance with its field steps."""

    def __init__(self, glasma, tau_start_fm=0.0, ox0=0.5, device="cuda"):
        self.glasma = glasma
        self.params = CorrParams(tau_start_fm, ox0)
        nb = lib().corr_workspace_bytes(C.byref(glasma.params))
        check(0 if nb >= 0 else nb)
        self._ws, ptr = _workspace(nb, device)
        h = C.c_void_p()
        check(lib().corr_create(glasma.handle, C.byref(self.params), C.c_void_p(ptr), nb, C.byref(h)))
        self.handle = h

    def table(self, cap=1 << 16):
        """Rows {tau_fm, static <dp_x^2>, <dp_y^2>, <dp_z^2>, lightlike <dp_x^2>, <dp_y^2>,
        <dp_z^2>} in GeV^2."""
        out = np.zeros((cap, 7))
        n = C.c_int64()
        check(lib().corr_table(self.handle, _dp(out), cap, C.byref(n)))
        return out[: n.value]

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            lib().corr_destroy(h)
            self.handle = None


class CPIC:
    """A particle ensemble bound to a Glasma context."""

    def __init__(self, glasma, n_particles, mass_GeV, tau_form_fm, p_min_GeV=0.0, p_max_GeV=0.0, init_kind=0,
                 q2=4.0, q3=10.0 / 3.0, bin_every=0, seed=2, device="cuda", integrator=0, substeps=1, interp=0):
        self.glasma = glasma
        self.params = CpicParams(n_particles, init_kind, mass_GeV, tau_form_fm, p_min_GeV, p_max_GeV, q2, q3,
                                 bin_every, integrator, substeps, interp, seed)
        nb = lib().cpic_workspace_bytes(C.byref(glasma.params), C.byref(self.params))
        check(0 if nb >= 0 else nb)
        self._ws, ptr = _workspace(nb, device)
        self.handle = cpic_create(glasma.handle, self.params, ptr, nb)
        self.np = n_particles

    def init(self):
        cpic_init(self.handle)

    def set_particles(self, x, y, eta, px, py, peta, Q, p0):
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (x, y, eta, px, py, peta, Q, p0)]
        check(lib().cpic_init_from_host(self.handle, *[_dp(a) for a in arrs]))

    def get_particles(self):
        n = self.np
        out = [np.zeros(n) for _ in range(6)] + [np.zeros((n, 8))]
        check(lib().cpic_get_particles(self.handle, *[_dp(a) for a in out]))
        return dict(zip(("x", "y", "eta", "px", "py", "peta", "Q"), out))

    def push(self, n_steps=1):
        cpic_push(self.handle, n_steps)

    def broadening(self):
        return broadening_accumulate(self.handle, 1 << 16)

    def export_state(self):
        """Checkpoint blob of the particles and their broadening sums (numpy uint8)."""
        nb = lib().cpic_state_bytes(self.handle)
        check(0 if nb >= 0 else nb)
        blob = np.empty(nb, dtype=np.uint8)
        check(lib().cpic_export_state(self.handle, blob.ctypes.data_as(C.c_void_p), nb))
        return blob

    def import_state(self, blob):
        blob = np.ascontiguousarray(blob, dtype=np.uint8)
        check(lib().cpic_import_state(self.handle, blob.ctypes.data_as(C.c_void_p), blob.size))

    def casimir_drift(self):
        out = np.zeros(2)
        check(lib().cpic_casimir_drift(self.handle, _dp(out)))
        return out

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            lib().cpic_destroy(h)
            self.handle = None


class Batch:
    """Many events (each a GlasmaParams + CpicParams pair) advanced together."""

    MODES = {"graph": 0, "persistent": 1, "per_event": 2, "eager": 3}

    def __init__(self, events, particles, device="cuda", stream=None):
        # a created stream of our own: the legacy default stream cannot be captured into a graph
        if stream is None:
            stream = torch.cuda.Stream(device=device)
        self.stream = stream
        E = len(events)
        self.ev = (GlasmaParams * E)(*events)
        self.pp = (CpicParams * E)(*particles)
        nb = lib().glasma_batch_workspace_bytes(self.ev, self.pp, E)
        check(0 if nb >= 0 else nb)
        self._ws, ptr = _workspace(nb, device)
        self.workspace_bytes = nb
        h = C.c_void_p()
        check(lib().glasma_batch_create(self.ev, self.pp, E, C.c_void_p(ptr), nb, _stream_ptr(stream), C.byref(h)))
        self.handle = h
        self.E = E

    def init(self):
        f = C.c_int64()
        check(lib().glasma_batch_init(self.handle, C.byref(f)))
        return f.value

    def run(self, mode="graph"):
        check(lib().glasma_batch_run(self.handle, self.MODES[mode]))

    def work(self):
        a, b = C.c_int64(), C.c_int64()
        check(lib().glasma_batch_work(self.handle, C.byref(a), C.byref(b)))
        return a.value, b.value

    def broadening(self, event):
        out = np.zeros((1 << 14, 5))
        n = C.c_int64()
        check(lib().glasma_batch_broadening(self.handle, event, _dp(out), out.shape[0], C.byref(n)))
        return out[: n.value]

    def diagnostics(self, event):
        out = np.zeros(8)
        check(lib().glasma_batch_diagnostics(self.handle, event, _dp(out)))
        return out

    def get_particles(self, event):
        n = self.pp[event].n_particles
        out = [np.zeros(n) for _ in range(6)] + [np.zeros((n, 8))]
        check(lib().glasma_batch_get_particles(self.handle, event, *[_dp(a) for a in out]))
        return dict(zip(("x", "y", "eta", "px", "py", "peta", "Q"), out))

    def state_bytes(self):
        return lib().glasma_batch_state_bytes(self.handle)

    def export_state(self, host_tensor):
        check(lib().glasma_batch_export_state(self.handle, C.c_void_p(host_tensor.data_ptr()), host_tensor.numel()))

    def import_state(self, host_tensor):
        check(lib().glasma_batch_import_state(self.handle, C.c_void_p(host_tensor.data_ptr()), host_tensor.numel()))

    def set_push_stream(self, separate=True):
        check(lib().glasma_batch_set_push_stream(self.handle, 1 if separate else 0))

    def set_wait_limit(self, polls=0):
        """glasma_batch_set_wait_limit: the persistent mode's grid-barrier wait in polls of
        ~100 ns (0: the default, ~2 s)."""
        check(lib().glasma_batch_set_wait_limit(self.handle, int(polls)))

    def set_graph_timing(self, on=True):
        check(lib().glasma_batch_set_graph_timing(self.handle, 1 if on else 0))

    def graph_times(self):
        """(field-kernel ms summed over the last run's launches, launches, span ms)."""
        f, n, sp = C.c_double(), C.c_int64(), C.c_double()
        check(lib().glasma_batch_graph_times(self.handle, C.byref(f), C.byref(n), C.byref(sp)))
        return f.value, n.value, sp.value

    def profile(self, mode="graph"):
        """CUDA-event timing of one eager run of the graph mode's launches: the batched field
        kernel (main) and the batched push (other)."""
        mm, om = C.c_double(), C.c_double()
        ml, ms, mp = C.c_int64(), C.c_int64(), C.c_int64()
        check(lib().glasma_batch_profile(self.handle, self.MODES[mode], C.byref(mm), C.byref(ml), C.byref(ms),
                                         C.byref(mp), C.byref(om)))
        return dict(main_ms=mm.value, main_launches=ml.value, main_sites=ms.value, main_particle_steps=mp.value,
                    other_ms=om.value)

    def launches(self, mode="graph"):
        return lib().glasma_batch_launches(self.handle, self.MODES[mode])

    @property
    def variant(self):
        return lib().glasma_batch_variant(self.handle)

    def set_variant(self, v):
        check(lib().glasma_batch_set_variant(self.handle, v))

    @property
    def push_variant(self):
        return lib().glasma_batch_push_variant(self.handle)

    def set_push_variant(self, v):
        check(lib().glasma_batch_set_push_variant(self.handle, v))

    def tune(self, steps=8):
        """glasma_batch_tune: time every field tile variant and every push kernel, keep the
        fastest of each.  Returns (chosen field variant, [ms per field variant]); the push
        kernel chosen is `push_variant`."""
        nv = lib().glasma_field_tile_variants(self.ev[0].precision)
        ms = (C.c_double * nv)()
        ch = C.c_int32()
        check(lib().glasma_batch_tune(self.handle, steps, C.byref(ch), ms))
        return ch.value, list(ms)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            lib().glasma_batch_destroy(h)
            self.handle = None


def push_many(ensembles, n_steps=1):
    """Coupled steps of several CPIC ensembles on one Glasma event (one field step, then
    each ensemble's push)."""
    cpic_push_many([c.handle for c in ensembles], n_steps)


def pool_broadening(table, group=None):
    """Pools the broadening tables of independent event replicas, one per rank of a
    torch.distributed group (Sec. 2: <dp_i^2> is an average over particles and events):
    every rank passes its table (rows {tau_fm, <dpx^2>, <dpy^2>, <dpz^2>, count} on the
    same tau grid) and gets the count-weighted average over all ranks, with the summed
    counts.  A host-side FP64 all-reduce of sums; the replicas exchange nothing else."""
    import torch
    import torch.distributed as dist

    t = np.asarray(table, dtype=np.float64)
    grid = torch.tensor([t.shape[0], t[:, 0].sum() if t.size else 0.0], dtype=torch.float64)
    lo, hi = grid.clone(), grid.clone()
    dist.all_reduce(lo, op=dist.ReduceOp.MIN, group=group)
    dist.all_reduce(hi, op=dist.ReduceOp.MAX, group=group)
    if not (torch.equal(lo, hi)):
        raise ValueError("broadening tables of the replicas are on different tau grids")
    w = torch.from_numpy(np.concatenate([t[:, 1:4] * t[:, 4:5], t[:, 4:5]], axis=1).copy())
    dist.all_reduce(w, group=group)
    w = w.numpy()
    out = t.copy()
    cnt = w[:, 3]
    out[:, 1:4] = np.where(cnt[:, None] > 0, w[:, :3] / np.where(cnt > 0, cnt, 1.0)[:, None], 0.0)
    out[:, 4] = cnt
    return out


def broadening_transport(table, kind="hq"):
    """Eq. 3 through the library's broadening_transport: rows {tau, d<dpx^2>/dtau,
    d<dpy^2>/dtau, d<dpz^2>/dtau, transverse, longitudinal, total, anisotropy}; kind "hq"
    (kappa_T, kappa_L, <dp_L^2>/<dp_T^2>) or "jet" (qhat_y, qhat_z, <dp_z^2>/<dp_y^2>)."""
    t = np.ascontiguousarray(table, dtype=np.float64)
    out = np.zeros((t.shape[0], 8))
    if t.shape[0] == 0:
        return out
    if kind not in ("hq", "jet"):
        raise ValueError("kind must be 'hq' or 'jet'")
    k = GLASMA_HEAVY_QUARKS if kind == "hq" else GLASMA_JETS_X
    check(lib().broadening_transport(_dp(t), t.shape[0], t.shape[1], k, _dp(out)))
    return out


def anisotropy(table, kind="hq"):
    """Rows {tau_fm, ratio}: <dp_L^2>/<dp_T^2> for heavy quarks, <dp_z^2>/<dp_y^2> for
    jets along x (NaN where the transverse broadening is zero); broadening_transport."""
    return broadening_transport(table, kind)[:, [0, 7]]


def kappa_qhat(table):
    """Rows {tau_fm, d<dpx^2>/dtau, d<dpy^2>/dtau, d<dpz^2>/dtau} (GeV^2/fm) of Eq. 3;
    broadening_transport."""
    return broadening_transport(table)[:, :4]


def field_tile_shape(precision, v):
    """(TX, TY, minimum CTAs per SM) of field tile variant v."""
    a, b, c = C.c_int32(), C.c_int32(), C.c_int32()
    check(lib().glasma_field_tile_shape(precision, v, C.byref(a), C.byref(b), C.byref(c)))
    return a.value, b.value, c.value


def field_tile_variants(precision):
    return lib().glasma_field_tile_variants(precision)
