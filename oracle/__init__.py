"""ctypes binding of the FP64 CPU oracle (test infrastructure).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import
this package.  Arrays follow the oracle's layout (see oracle.h):
U complex128[N*N, 2, 3, 3], E float64[N*N, 2, 8], phi/pi float64[N*N, 8],
site index s = x + N*y.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = C.CDLL(path)
        _declare(_lib)
    return _lib


_d = C.c_double
_i = C.c_int
_p = C.c_void_p
_u64 = C.c_uint64


def _declare(L):
    sig = {
        "o_generator": (None, [_i, _p]),
        "o_alg_to_mat": (None, [_p, _p]),
        "o_mat_to_alg": (None, [_p, _p]),
        "o_im_tl": (None, [_p, _p]),
        "o_exp_i": (None, [_p, _p]),
        "o_expm": (None, [_p, _p]),
        "o_transport": (None, [_p, _p, _p]),
        "o_conj_by": (None, [_p, _p, _p]),
        "o_structure_constants": (None, [_p, _p]),
        "o_haar": (None, [_p, _p]),
        "o_reunitarize": (None, [_p]),
        "o_unitarity_dev": (_d, [_p]),
        "o_philox4x32_10": (None, [_p, _p, _p]),
        "o_fft2": (_i, [_i, _p, _i]),
        "o_mv_charges": (None, [_i, _i, _d, _u64, _i, _i, _p]),
        "o_poisson": (_i, [_i, _d, _p, _p]),
        "o_wilson_line": (_i, [_i, _i, _d, _d, _u64, _i, _p]),
        "o_pure_gauge_links": (None, [_i, _p, _p]),
        "o_ic_residual": (None, [_p, _p, _p, _p]),
        "o_ic_jacobian": (None, [_p, _p, _p, _p]),
        "o_ic_solve_link": (_i, [_p, _p, _p, _d, _i, _p]),
        "o_ic_solve": (_i, [_i, _p, _p, _p, _d, _i, _p, _p, _p]),
        "o_pi0": (None, [_i, _p, _p, _p, _p]),
        "o_glasma_init": (_i, [_i, _i, _d, _d, _u64, _d, _d, _i, _p, _p, _p, _p, _p]),
        "o_potential": (_d, [_i, _d, _i, _p, _p]),
        "o_force": (None, [_i, _d, _i, _p, _p, _p, _p]),
        "o_field_step": (None, [_i, _i, _d, _i, _p, _p, _p, _p, _p, _p, _p, _p]),
        "o_reunitarize_all": (None, [_i, _p]),
        "o_gauss": (None, [_i, _p, _p, _p, _p, _p]),
        "o_gauss_rel": (_d, [_i, _p, _p, _p, _p]),
        "o_energy": (None, [_i, _d, _i, _p, _p, _p, _p, _p]),
        "o_unitarity_all": (_d, [_i, _p]),
        "o_particles_init": (None, [_i, _i, _d, _i, _d, _d, _d, _d, _u64] + [_p] * 7),
        "o_q0_cartan": (None, [_d, _d, _p]),
        "o_gather": (None, [_i, _d, _i, _p, _p, _p, _p, _p, _p, _i, _i, _p]),
        "o_corr_step": (None, [_i, _i, _d, _i] + [_p] * 9 + [_i, _i, _p]),
        "o_push": (None, [_i, _i, _i, _d, _i, _d] + [_p] * 6 + [_p] * 7 + [_p, _p]),
        "o_push_int": (None, [_i, _i, _i, _d, _i, _d] + [_p] * 6 + [_p] * 7 + [_p, _p, _i]),
        "o_set_threads": (_i, [_i]),
        "o_push_sub": (None, [_i, _i, _i, _d, _i, _d] + [_p] * 6 + [_p] * 7 + [_p, _p, _i, _i]),
        "o_push_ext": (None, [_i, _i, _i, _d, _i, _d] + [_p] * 6 + [_p] * 7 + [_p, _p, _i, _i, _i]),
        "o_gather_cic": (None, [_i, _d, _i] + [_p] * 6 + [_i, _i, _d, _d, _p]),
        "o_casimirs": (None, [_p, _p, _p]),
        "o_derivative": (None, [_i, _p, _i, _p, _i, _p, _i]),
        "o_transport_coefficients": (None, [_i, _p, _i, _i, _p]),
        "o_pz_lab": (_d, [_d, _d, _d, _d, _d]),
        "o_mlp_forward": (None, [_i] + [_p] * 10),
        "o_mlp_loss_backward": (_d, [_i] + [_p] * 14),
        "o_ic_features": (None, [_p, _p, _p]),
        "o_ic_target": (None, [_p, _p, _p, _p]),
        "o_ic_delta": (None, [_p, _p, _p, _p]),
        "o_ic_series": (None, [_p, _p, _p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def _ptr(a):
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    return a.ctypes.data


def cz(*shape):
    return np.zeros(shape, dtype=np.complex128)


def rz(*shape):
    return np.zeros(shape, dtype=np.float64)


# ---------------------------------------------------------------- su(3)
def generator(a):
    T = cz(3, 3)
    lib().o_generator(a, _ptr(T))
    return T


def alg_to_mat(x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    X = cz(3, 3)
    lib().o_alg_to_mat(_ptr(x), _ptr(X))
    return X


def mat_to_alg(X):
    X = np.ascontiguousarray(X, dtype=np.complex128)
    x = rz(8)
    lib().o_mat_to_alg(_ptr(X), _ptr(x))
    return x


def im_tl(P):
    P = np.ascontiguousarray(P, dtype=np.complex128)
    x = rz(8)
    lib().o_im_tl(_ptr(P), _ptr(x))
    return x


def exp_i(x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    U = cz(3, 3)
    lib().o_exp_i(_ptr(x), _ptr(U))
    return U


def expm(A):
    A = np.ascontiguousarray(A, dtype=np.complex128)
    R = cz(3, 3)
    lib().o_expm(_ptr(A), _ptr(R))
    return R


def transport(U, x):
    U = np.ascontiguousarray(U, dtype=np.complex128)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = rz(8)
    lib().o_transport(_ptr(U), _ptr(x), _ptr(y))
    return y


def conj_by(U, x):
    U = np.ascontiguousarray(U, dtype=np.complex128)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = rz(8)
    lib().o_conj_by(_ptr(U), _ptr(x), _ptr(y))
    return y


def structure_constants():
    f = rz(8, 8, 8)
    d = rz(8, 8, 8)
    lib().o_structure_constants(_ptr(f), _ptr(d))
    return f, d


def haar(g18):
    g = np.ascontiguousarray(g18, dtype=np.float64)
    U = cz(3, 3)
    lib().o_haar(_ptr(g), _ptr(U))
    return U


def reunitarize(U):
    U = np.array(U, dtype=np.complex128, order="C")
    lib().o_reunitarize(_ptr(U))
    return U


def unitarity_dev(U):
    U = np.ascontiguousarray(U, dtype=np.complex128)
    return lib().o_unitarity_dev(_ptr(U))


# ---------------------------------------------------------------- rng / fft
def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().o_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def fft2(a, sign=-1):
    a = np.array(a, dtype=np.complex128, order="C")
    assert lib().o_fft2(a.shape[0], _ptr(a), sign) == 0
    return a


# ---------------------------------------------------------------- initial conditions
def mv_charges(n, n_sheets, g2mua, seed, nucleus, sheet):
    rho = rz(n * n, 8)
    lib().o_mv_charges(n, n_sheets, g2mua, seed, nucleus, sheet, _ptr(rho))
    return rho


def poisson(n, m2, rho):
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    lam = rz(n * n, 8)
    assert lib().o_poisson(n, m2, _ptr(rho), _ptr(lam)) == 0
    return lam


def wilson_line(n, n_sheets, g2mua, m_ir_a, seed, nucleus):
    V = cz(n * n, 3, 3)
    assert lib().o_wilson_line(n, n_sheets, g2mua, m_ir_a, seed, nucleus, _ptr(V)) == 0
    return V


def pure_gauge_links(n, V):
    V = np.ascontiguousarray(V, dtype=np.complex128)
    UA = cz(n * n, 2, 3, 3)
    lib().o_pure_gauge_links(n, _ptr(V), _ptr(UA))
    return UA


def ic_residual(U1, U2, U):
    r = rz(8)
    args = [np.ascontiguousarray(m, dtype=np.complex128) for m in (U1, U2, U)]
    lib().o_ic_residual(*[_ptr(m) for m in args], _ptr(r))
    return r


def ic_jacobian(U1, U2, U):
    J = rz(8, 8)
    args = [np.ascontiguousarray(m, dtype=np.complex128) for m in (U1, U2, U)]
    lib().o_ic_jacobian(*[_ptr(m) for m in args], _ptr(J))
    return J


def ic_solve_link(U1, U2, U_start=None, tol=1e-12, max_iter=100):
    U = np.eye(3, dtype=np.complex128) if U_start is None else np.array(U_start, dtype=np.complex128)
    res = np.zeros(1)
    a1 = np.ascontiguousarray(U1, dtype=np.complex128)
    a2 = np.ascontiguousarray(U2, dtype=np.complex128)
    it = lib().o_ic_solve_link(_ptr(a1), _ptr(a2), _ptr(U), tol, max_iter, _ptr(res))
    return U, it, res[0]


def ic_solve(n, U1, U2, U_start=None, tol=1e-12, max_iter=100):
    U = cz(n * n, 2, 3, 3)
    iters = np.zeros(2 * n * n, dtype=np.int32)
    res = rz(2 * n * n)
    a1 = np.ascontiguousarray(U1, dtype=np.complex128)
    a2 = np.ascontiguousarray(U2, dtype=np.complex128)
    st = None if U_start is None else np.ascontiguousarray(U_start, dtype=np.complex128)
    fails = lib().o_ic_solve(n, _ptr(a1), _ptr(a2), None if st is None else _ptr(st), tol,
                             max_iter, _ptr(U), _ptr(iters), _ptr(res))
    return U, iters, res, fails


def pi0(n, U, U1, U2):
    pi = rz(n * n, 8)
    args = [np.ascontiguousarray(m, dtype=np.complex128) for m in (U, U1, U2)]
    lib().o_pi0(n, *[_ptr(m) for m in args], _ptr(pi))
    return pi


class State:
    """Field state at step n: U, phi at tau_n; E, pi at tau_{n-1/2}."""

    def __init__(self, n, step=1):
        self.n = n
        self.step = step
        self.U = cz(n * n, 2, 3, 3)
        self.E = rz(n * n, 2, 8)
        self.phi = rz(n * n, 8)
        self.pi = rz(n * n, 8)

    def copy(self):
        s = State(self.n, self.step)
        s.U[...] = self.U
        s.E[...] = self.E
        s.phi[...] = self.phi
        s.pi[...] = self.pi
        return s


def glasma_init(n, n_sheets, g2mua, m_ir_a, seed, dtau, tol=1e-12, max_iter=100):
    st = State(n, step=1)
    iters = np.zeros(2 * n * n, dtype=np.int32)
    fails = lib().o_glasma_init(n, n_sheets, g2mua, m_ir_a, seed, dtau, tol, max_iter,
                                _ptr(st.U), _ptr(st.E), _ptr(st.phi), _ptr(st.pi), _ptr(iters))
    return st, iters, fails


# ---------------------------------------------------------------- field
def potential(n, tau, expanding, U, phi):
    return lib().o_potential(n, tau, expanding, _ptr(U), _ptr(phi))


def force(n, tau, expanding, U, phi):
    fE = rz(n * n, 2, 8)
    fpi = rz(n * n, 8)
    lib().o_force(n, tau, expanding, _ptr(U), _ptr(phi), _ptr(fE), _ptr(fpi))
    return fE, fpi


def field_step(st, dtau, expanding=1):
    n = st.n
    nx = State(n, st.step + 1)
    lib().o_field_step(n, expanding, dtau, st.step, _ptr(st.U), _ptr(st.E), _ptr(st.phi),
                       _ptr(st.pi), _ptr(nx.U), _ptr(nx.E), _ptr(nx.phi), _ptr(nx.pi))
    return nx


def reunitarize_all(st):
    lib().o_reunitarize_all(st.n, _ptr(st.U))


def gauss(st):
    G = rz(st.n * st.n, 8)
    lib().o_gauss(st.n, _ptr(st.U), _ptr(st.E), _ptr(st.phi), _ptr(st.pi), _ptr(G))
    return G


def gauss_rel(st):
    return lib().o_gauss_rel(st.n, _ptr(st.U), _ptr(st.E), _ptr(st.phi), _ptr(st.pi))


def energy(n, tau, expanding, U, E, phi, pi):
    out = rz(4)
    E = np.ascontiguousarray(E)
    pi = np.ascontiguousarray(pi)
    lib().o_energy(n, tau, expanding, _ptr(U), _ptr(E), _ptr(phi), _ptr(pi), _ptr(out))
    return out


def unitarity_all(st):
    return lib().o_unitarity_all(st.n, _ptr(st.U))


# ---------------------------------------------------------------- particles
class Particles:
    def __init__(self, np_):
        self.np = np_
        self.x = rz(np_)
        self.y = rz(np_)
        self.eta = rz(np_)
        self.px = rz(np_)
        self.py = rz(np_)
        self.peta = rz(np_)
        self.Q = rz(np_, 8)
        self.p0 = rz(np_, 3)

    def copy(self):
        o = Particles(self.np)
        for k in ("x", "y", "eta", "px", "py", "peta", "Q", "p0"):
            getattr(o, k)[...] = getattr(self, k)
        return o

    def set_p0(self, mass, expanding=1):
        self.p0[:, 0] = self.px
        self.p0[:, 1] = self.py
        if expanding:
            self.p0[:, 2] = [pz_lab(mass, a, b, c, e)
                             for a, b, c, e in zip(self.px, self.py, self.peta, self.eta)]
        else:
            self.p0[:, 2] = self.peta


def particles_init(np_, n, mass, init_kind, p_min, p_max, seed, q2=4.0, q3=10.0 / 3.0):
    P = Particles(np_)
    lib().o_particles_init(np_, n, mass, init_kind, p_min, p_max, q2, q3, seed, _ptr(P.x),
                           _ptr(P.y), _ptr(P.eta), _ptr(P.px), _ptr(P.py), _ptr(P.peta),
                           _ptr(P.Q))
    P.set_p0(mass)
    return P


def q0_cartan(q2=4.0, q3=10.0 / 3.0):
    q = rz(8)
    lib().o_q0_cartan(q2, q3, _ptr(q))
    return q


def gather(old, new, cx, cy, dtau, expanding=1):
    """Site-centred (Ex, Ey, Ez, Bx, By, Bz) at cell (cx, cy) for the push of step old.step."""
    F = rz(6, 8)
    tau = old.step * dtau
    lib().o_gather(old.n, tau, expanding, _ptr(old.U), _ptr(old.E), _ptr(new.E), _ptr(old.phi),
                   _ptr(old.pi), _ptr(new.pi), cx, cy, _ptr(F))
    return F


class Correlators:
    """Running static (Eq. 4) and lightlike (Eq. 5) estimators of one event (correlators.c),
    started at the step of the first call; the lightlike paths start at offset ox0 in
    their cells."""

    def __init__(self, n, ox0=0.5):
        self.n, self.ox0, self.m = n, ox0, 0
        self.Istat = rz(n * n, 3, 8)
        self.W = np.ascontiguousarray(np.broadcast_to(np.eye(3, dtype=np.complex128), (n * n, 3, 3)))
        self.J = rz(n * n, 3, 8)

    def crossings(self, m, dtau):
        return int(np.floor(self.ox0 + m * dtau))

    def step(self, old, new, dtau, expanding=1):
        """One step (old: the fields of step n, new: of step n+1); returns the static
        <dp_x^2>, <dp_y^2>, <dp_z^2> and the lightlike ones, in lattice units."""
        out = rz(6)
        k0, k1 = self.crossings(self.m, dtau), self.crossings(self.m + 1, dtau)
        lib().o_corr_step(self.n, expanding, dtau, old.step, _ptr(old.U), _ptr(old.E), _ptr(new.E), _ptr(old.phi),
                          _ptr(old.pi), _ptr(new.pi), _ptr(self.Istat), _ptr(self.W), _ptr(self.J), k0, k1,
                          _ptr(out))
        self.m += 1
        return out


def push(P, old, new, dtau, mass, expanding=1, integrator=0, substeps=1, interp=0):
    """One push of step old.step -> old.step+1 (old: fields before, new: after the field step);
    integrator 0 explicit, 1 Boris; substeps particle steps of dtau / substeps; interp 0
    nearest grid point, 1 cloud in cell."""
    acc = rz(4)
    lib().o_push_ext(P.np, old.n, expanding, dtau, old.step, mass, _ptr(old.U), _ptr(old.E),
                     _ptr(new.E), _ptr(old.phi), _ptr(old.pi), _ptr(new.pi), _ptr(P.x), _ptr(P.y),
                     _ptr(P.eta), _ptr(P.px), _ptr(P.py), _ptr(P.peta), _ptr(P.Q), _ptr(P.p0),
                     _ptr(acc), integrator, substeps, interp)
    return acc


def gather_cic(old, new, cx, cy, ox, oy, dtau, expanding=1):
    """Cloud-in-cell (Ex, Ey, Ez, Bx, By, Bz) for offsets (ox, oy) in cell (cx, cy), in the
    frame of site (cx, cy), for the push of step old.step."""
    F = rz(6, 8)
    tau = old.step * dtau
    lib().o_gather_cic(old.n, tau, expanding, _ptr(old.U), _ptr(old.E), _ptr(new.E), _ptr(old.phi),
                       _ptr(old.pi), _ptr(new.pi), cx, cy, ox, oy, _ptr(F))
    return F


def casimirs(Q):
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    a = np.zeros(1)
    b = np.zeros(1)
    lib().o_casimirs(_ptr(Q), _ptr(a), _ptr(b))
    return a[0], b[0]


def pz_lab(mass, px, py, peta, eta):
    return lib().o_pz_lab(mass, px, py, peta, eta)


# ---------------------------------------------------------------- Eq. 3 estimators
def derivative(tau, f):
    """d f / d tau on the grid tau: central differences inside, one-sided at the ends."""
    tau = np.ascontiguousarray(tau, dtype=np.float64)
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros(len(tau))
    lib().o_derivative(len(tau), _ptr(tau), 1, _ptr(f), 1, _ptr(out), 1)
    return out


def transport_coefficients(table, kind="hq"):
    """Eq. 3 on a broadening table (rows {tau, <dpx^2>, <dpy^2>, <dpz^2>, ...}): rows
    {tau, d<dpx^2>/dtau, d<dpy^2>/dtau, d<dpz^2>/dtau, transverse, longitudinal, total,
    anisotropy}; kind "hq" (kappa_T, kappa_L, <dp_L^2>/<dp_T^2>) or "jet" (qhat_y, qhat_z,
    <dp_z^2>/<dp_y^2>)."""
    t = np.ascontiguousarray(table, dtype=np.float64)
    out = np.zeros((t.shape[0], 8))
    lib().o_transport_coefficients(t.shape[0], _ptr(t), t.shape[1], 0 if kind == "hq" else 1, _ptr(out))
    return out


def kappa_qhat(table):
    """Rows {tau, d<dpx^2>/dtau, d<dpy^2>/dtau, d<dpz^2>/dtau} of Eq. 3."""
    return transport_coefficients(table)[:, :4]


# ---------------------------------------------------------------- warm-start network
MLP_SHAPES = {"W1": (128, 36), "b1": (128,), "W2": (128, 128), "b2": (128,), "W3": (16, 128), "b3": (16,)}


def mlp_forward(x, w):
    x = np.ascontiguousarray(x, dtype=np.float64)
    B = x.shape[0]
    h1, h2, y = rz(B, 128), rz(B, 128), rz(B, 16)
    ws = [np.ascontiguousarray(w[k], dtype=np.float64) for k in ("W1", "b1", "W2", "b2", "W3", "b3")]
    lib().o_mlp_forward(B, _ptr(x), *[_ptr(a) for a in ws], _ptr(h1), _ptr(h2), _ptr(y))
    return y, h1, h2


def mlp_loss_grad(x, t, w):
    x = np.ascontiguousarray(x, dtype=np.float64)
    t = np.ascontiguousarray(t, dtype=np.float64)
    ws = [np.ascontiguousarray(w[k], dtype=np.float64) for k in ("W1", "b1", "W2", "b2", "W3", "b3")]
    g = {k: rz(*s) for k, s in MLP_SHAPES.items()}
    loss = lib().o_mlp_loss_backward(x.shape[0], _ptr(x), _ptr(t), *[_ptr(a) for a in ws],
                                     *[_ptr(g[k]) for k in ("W1", "b1", "W2", "b2", "W3", "b3")])
    return loss, g


def ic_features(U1, U2):
    f = rz(36)
    a = np.ascontiguousarray(U1, dtype=np.complex128)
    b = np.ascontiguousarray(U2, dtype=np.complex128)
    lib().o_ic_features(_ptr(a), _ptr(b), _ptr(f))
    return f


def ic_series(U1, U2):
    d = rz(8)
    args = [np.ascontiguousarray(m, dtype=np.complex128) for m in (U1, U2)]
    lib().o_ic_series(*[_ptr(m) for m in args], _ptr(d))
    return d


def ic_delta(U1, U2, U):
    d = rz(8)
    args = [np.ascontiguousarray(m, dtype=np.complex128) for m in (U1, U2, U)]
    lib().o_ic_delta(*[_ptr(m) for m in args], _ptr(d))
    return d


def ic_target(U1, U2, U):
    d = rz(8)
    args = [np.ascontiguousarray(m, dtype=np.complex128) for m in (U1, U2, U)]
    lib().o_ic_target(*[_ptr(m) for m in args], _ptr(d))
    return d


def set_threads(n):
    """OpenMP threads of the oracle's loops (n <= 0: query); returns the count in effect."""
    return lib().o_set_threads(n)
