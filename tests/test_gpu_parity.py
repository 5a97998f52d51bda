"""GPU-vs-oracle parity through the C ABI (libglasma.so).

FP64 mode: 1e-10 relative (normwise per field / per observable).  FP32 mode:
the tolerance follows from the arithmetic: one FP32 step carries ~1e-7
relative rounding per operation; a few tens of SU(3) products per site and
step give ~1e-6 per step, growing at most linearly over the few steps
compared here, so 2e-5 bounds a 10-step comparison.
"""
import numpy as np
import pytest

import oracle as O
from gpu_common import HBARC, lattice_units, random_particles, random_state, rel_err

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_2307_07999_gb300")


def gpu_fields(n, prec, expanding=1, tau_end=100.0, L=6.0, **kw):
    return G.Glasma(n, L, precision=prec, expanding=expanding, tau_end_fm=tau_end, **kw)


def compare_states(g, st, tol):
    U, E, phi, pi, step = g.get_state()
    assert step == st.step
    errs = dict(U=rel_err(U, st.U), E=rel_err(E, st.E), phi=rel_err(phi, st.phi), pi=rel_err(pi, st.pi))
    for k, v in errs.items():
        assert v < tol, (k, v, errs)
    return errs


@pytest.mark.parametrize("n", [2, 8, 37, 64])
@pytest.mark.parametrize("expanding", [1, 0])
def test_field_steps_fp64(n, expanding):
    st = random_state(n, seed=100 + n, step=3)
    g = gpu_fields(n, 0, expanding)
    g.set_state(st.U, st.E, st.phi, st.pi, st.step)
    for _ in range(6):
        st = O.field_step(st, 0.125, expanding)
    g.step(6)
    compare_states(g, st, 1e-10)


@pytest.mark.parametrize("n", [8, 37, 64])
def test_field_steps_fp32(n):
    st = random_state(n, seed=200 + n, step=3)
    g = gpu_fields(n, 1)
    g.set_state(st.U, st.E, st.phi, st.pi, st.step)
    for _ in range(10):
        st = O.field_step(st, 0.125, 1)
    g.step(10)
    compare_states(g, st, 2e-5)


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_stored_plaquettes(prec, tol):
    """The one-event field step stores, in the eighth plane group of the buffer it reads, ImTL
    of every site's plaquette U_x(x) U_y(x+x) U_x(x+y)^dag U_y(x)^dag of that buffer's
    links (the push of the step reads them).  A context rotates two buffers, so the buffer
    a checkpoint exports two steps on is the one the first step read."""
    n = 8
    st = random_state(n, seed=414, step=3)
    g = gpu_fields(n, prec)
    g.set_state(st.U, st.E, st.phi, st.pi, st.step)
    g.step(2)
    blob = g.export_state()
    rs = 4 if prec else 8
    body_bytes = (64 * n * n * rs + 255) // 256 * 256
    body = blob[blob.size - body_bytes: blob.size - body_bytes + 64 * n * n * rs]
    F = body.view(np.float32 if prec else np.float64).reshape(8, n * n, 8)[7].astype(np.float64)
    want = np.zeros((n * n, 8))
    for y in range(n):
        for x in range(n):
            s = x + n * y
            sx, sy = (x + 1) % n + n * y, x + n * ((y + 1) % n)
            P = st.U[s, 0] @ st.U[sx, 1] @ st.U[sy, 0].conj().T @ st.U[s, 1].conj().T
            want[s] = O.im_tl(P)
    assert rel_err(F, want) < tol


def test_reunitarisation_fp32_keeps_links_unitary():
    n = 32
    st = random_state(n, seed=7, step=3)
    g = gpu_fields(n, 1, reunit_every=4)
    g.set_state(st.U, st.E, st.phi, st.pi, st.step)
    g.step(40)
    d = g.diagnostics()
    assert d[5] < 2e-6


@pytest.mark.parametrize("n,L,tol", [(16, 6.0, 1e-12), (32, 6.0, 1e-12), (32, 3.0, 1e-14), (48, 10.0, 1e-14)])
def test_initial_conditions_fp64(n, L, tol):
    """MV charges, Poisson, Wilson lines and the tau = 0+ Newton solve.  The number of
    Newton iterations is an integer decided by FP64 comparisons of two different
    rounding paths, and at strong coupling (g^2 mu a ~ 2-4) a link may settle on a
    different (equally valid) root; so: the GPU links must solve the matching
    condition to tol, the failures and iteration counts must agree in aggregate, and
    the links converged on both sides must agree to 1e-10 for at least 99% of them
    (all of them at weak coupling)."""
    a_fm, a, g2mua, mira = lattice_units(n, L)
    st, iters, fails = O.glasma_init(n, 10, g2mua, mira, 4242, 0.125, tol=tol)
    g = gpu_fields(n, 0, L=L, seed=4242, newton_tol=tol)
    gf, gmean, gmax = g.init()
    assert abs(gf - fails) <= max(1, fails // 10)
    assert abs(gmean - iters[iters >= 0].mean()) < 0.05 * iters[iters >= 0].mean()
    U, E, phi, pi, step = g.get_state()
    assert step == 1 and np.all(E == 0)
    V1 = O.wilson_line(n, 10, g2mua, mira, 4242, 0)
    V2 = O.wilson_line(n, 10, g2mua, mira, 4242, 1)
    U1, U2 = O.pure_gauge_links(n, V1), O.pure_gauge_links(n, V2)
    conv = iters.reshape(n * n, 2) >= 0
    res = np.array([[np.linalg.norm(O.ic_residual(U1[s, d], U2[s, d], U[s, d])) for d in range(2)]
                    for s in range(n * n)])
    # the residual re-evaluated on the other side carries ~1e-14 of FP64 rounding
    assert np.mean(res <= tol + 3e-14) >= np.mean(conv) - 0.01
    same = np.abs(U - st.U).reshape(n * n, 2, -1).max(-1) < 1e-10
    frac = same[conv].mean()
    if g2mua < 1.2:
        assert frac == 1.0
        assert rel_err(pi, st.pi) < 1e-10 and rel_err(phi, st.phi) < 1e-10
    else:
        assert frac >= 0.99


def test_particle_init_matches_oracle():
    n, np_ = 32, 4000
    a_fm, a, g2mua, mira = lattice_units(n, 6.0)
    g = gpu_fields(n, 0)
    st = random_state(n, seed=1, step=2)
    g.set_state(st.U, st.E, st.phi, st.pi, st.step)
    c = G.CPIC(g, np_, 1.5, 0.1, p_min_GeV=0.0, p_max_GeV=5.0, init_kind=0, seed=99)
    c.init()
    P = O.particles_init(np_, n, 1.5 * a, 0, 0.0, 5.0 * a, 99)
    got = c.get_particles()
    assert np.abs(got["x"] - P.x).max() < 1e-12 and np.abs(got["y"] - P.y).max() < 1e-12
    assert np.abs(got["px"] - P.px).max() < 1e-12 and np.abs(got["py"] - P.py).max() < 1e-12
    assert np.abs(got["Q"] - P.Q).max() < 1e-12


def run_pair(n, np_, steps, prec, seed, expanding=1, mass=0.5, bin_every=0):
    st = random_state(n, seed=seed, step=4)
    P = random_particles(np_, n, seed + 1, mass=mass)
    g = gpu_fields(n, prec, expanding)
    g.set_state(st.U, st.E, st.phi, st.pi, st.step)
    a_gev = (6.0 / n) / HBARC
    c = G.CPIC(g, np_, mass / a_gev, 0.0, bin_every=bin_every)
    c.set_particles(P.x, P.y, P.eta, P.px, P.py, P.peta, P.Q, P.p0)
    accs = []
    for _ in range(steps):
        nx = O.field_step(st, 0.125, expanding)
        accs.append(O.push(P, st, nx, 0.125, mass, expanding))
        st = nx
    c.push(steps)
    return g, c, st, P, np.array(accs), a_gev


@pytest.mark.parametrize("expanding", [1, 0])
def test_push_fp64(expanding):
    n, np_ = 12, 300
    g, c, st, P, accs, a_gev = run_pair(n, np_, 12, 0, 31, expanding)
    got = c.get_particles()
    dx = np.abs(got["x"] - P.x)
    dy = np.abs(got["y"] - P.y)
    assert np.minimum(dx, n - dx).max() < 1e-10 and np.minimum(dy, n - dy).max() < 1e-10
    for k in ("px", "py", "peta", "eta"):
        assert rel_err(got[k], getattr(P, k)) < 1e-10, k
    assert rel_err(got["Q"], P.Q) < 1e-10
    tab = c.broadening()
    want = accs[:, :3] / accs[:, 3:4] / a_gev ** 2
    assert rel_err(tab[1:, 1:4], want) < 1e-10
    assert np.all(tab[1:, 4] == np_)


def test_push_sorting_is_invisible():
    n, np_ = 16, 500
    _, c1, _, _, _, _ = run_pair(n, np_, 10, 0, 41, bin_every=0)
    _, c2, _, _, _, _ = run_pair(n, np_, 10, 0, 41, bin_every=3)
    a, b = c1.get_particles(), c2.get_particles()
    for k in a:
        assert np.abs(a[k] - b[k]).max() < 1e-13, k
    assert rel_err(c2.broadening()[:, 1:4], c1.broadening()[:, 1:4]) < 1e-13


@pytest.mark.parametrize("prec,bin_every,tol", [(0, 3, 1e-10), (0, 1, 1e-10), (1, 2, 1e-4)])
def test_push_sorted_matches_oracle(prec, bin_every, tol):
    """Particles sorted by cell every k steps (a counting sort that reorders the particle
    planes; results are reported in the original order) against the oracle, which keeps
    its particles unsorted."""
    n, np_ = 16, 600
    g, c, st, P, accs, a_gev = run_pair(n, np_, 14, prec, 43, bin_every=bin_every)
    got = c.get_particles()
    dx = np.abs(got["x"] - P.x)
    dy = np.abs(got["y"] - P.y)
    assert np.minimum(dx, n - dx).max() < tol * n and np.minimum(dy, n - dy).max() < tol * n
    for k in ("px", "py", "peta", "eta"):
        assert rel_err(got[k], getattr(P, k)) < tol, k
    assert rel_err(got["Q"], P.Q) < tol
    tab = c.broadening()
    want = accs[:, :3] / accs[:, 3:4] / a_gev ** 2
    assert rel_err(tab[1:, 1:4], want) < tol
    assert np.all(tab[1:, 4] == np_)


def test_push_massless_and_empty():
    n = 10
    g, c, st, P, accs, a_gev = run_pair(n, 64, 6, 0, 51, mass=0.0)
    got = c.get_particles()
    assert rel_err(got["px"], P.px) < 1e-10
    g2 = gpu_fields(n, 0)
    st2 = random_state(n, seed=3, step=4)
    g2.set_state(st2.U, st2.E, st2.phi, st2.pi, 4)
    c2 = G.CPIC(g2, 0, 1.0, 0.0)
    c2.init()
    c2.push(3)
    tab = c2.broadening()
    assert np.all(tab[:, 1:4] == 0)


_CONFIG1 = {}


def config1_oracle(n=32, L=6.0, np_=1000, mass_gev=1.5, tau_form=0.1, seed=12345, pseed=777):
    """The oracle's run of the 32^2 configuration: broadening table and the initial
    state at step 1 (uploaded to the GPU so that both sides evolve the same fields)."""
    key = (n, L, np_, mass_gev, tau_form, seed, pseed)
    if key in _CONFIG1:
        return _CONFIG1[key]
    a_fm, a, g2mua, mira = lattice_units(n, L)
    st, iters, fails = O.glasma_init(n, 10, g2mua, mira, seed, 0.125)
    st0 = st.copy()
    P = O.particles_init(np_, n, mass_gev * a, 0, 0.0, 0.0, pseed)
    nform = int(round(tau_form / (0.125 * a_fm)))
    nsteps = int(np.ceil(1.0 / (0.125 * a_fm) - 1e-9))
    while st.step < nform:
        st = O.field_step(st, 0.125)
    rows = [(nform * 0.125 * a_fm, 0.0, 0.0, 0.0, np_)]
    while st.step < nsteps:
        nx = O.field_step(st, 0.125)
        acc = O.push(P, st, nx, 0.125, mass_gev * a)
        rows.append((nx.step * 0.125 * a_fm, *(acc[:3] / acc[3] / a ** 2), acc[3]))
        st = nx
    _CONFIG1[key] = (np.array(rows), st0)
    return _CONFIG1[key]


def test_config1_broadening_fp64():
    """32^2, L = 6 fm, g^2 mu = 2 GeV, m = 0.2 GeV, 10 sheets, 1000 charm (1.5 GeV, p = 0,
    tau_form = 0.1 fm/c) to tau = 1 fm/c: <dp_i^2>(tau) and kappa at 1e-10."""
    want, st0 = config1_oracle()
    g = gpu_fields(32, 0, L=6.0, tau_end=1.0, seed=12345)
    g.set_state(st0.U, st0.E, st0.phi, st0.pi, 1)
    c = G.CPIC(g, 1000, 1.5, 0.1, seed=777)
    c.init()
    n_form = int(round(0.1 / (0.125 * 6.0 / 32)))
    g.step(n_form - 1)
    c.push(int(np.ceil(1.0 / (0.125 * 6.0 / 32) - 1e-9)) - n_form)
    tab = c.broadening()
    assert tab.shape == want.shape
    assert np.abs(tab[:, 0] - want[:, 0]).max() < 1e-12
    assert rel_err(tab[:, 1:4], want[:, 1:4]) < 1e-10
    k_gpu, k_ref = G.kappa_qhat(tab), O.kappa_qhat(want)
    assert rel_err(k_gpu[:, 1:], k_ref[:, 1:]) < 1e-10
    drift = c.casimir_drift()
    assert drift[0] < 1e-11 and drift[1] < 1e-11


def test_config1_broadening_fp32_tolerance():
    """FP32 evolution against the FP64 oracle: <dp^2>(tau) and kappa within 1e-4 of the
    largest value, Gauss-law violation below 1e-5."""
    want, st0 = config1_oracle()
    g = gpu_fields(32, 1, L=6.0, tau_end=1.0, seed=12345, reunit_every=8)
    g.set_state(st0.U, st0.E, st0.phi, st0.pi, 1)
    c = G.CPIC(g, 1000, 1.5, 0.1, seed=777)
    c.init()
    n_form = int(round(0.1 / (0.125 * 6.0 / 32)))
    g.step(n_form - 1)
    c.push(int(np.ceil(1.0 / (0.125 * 6.0 / 32) - 1e-9)) - n_form)
    tab = c.broadening()
    e_dp = rel_err(tab[:, 1:4], want[:, 1:4])
    e_k = rel_err(G.kappa_qhat(tab)[:, 1:], O.kappa_qhat(want)[:, 1:])
    d = g.diagnostics()
    print("fp32 errors: dp2", e_dp, "kappa", e_k, "gauss", d[0], "unitarity", d[5])
    assert d[0] < 1e-5
    assert e_dp < 1e-4 and e_k < 1e-4


def test_monitors_match_oracle():
    n = 24
    st = random_state(n, seed=5, step=6)
    g = gpu_fields(n, 0)
    g.set_state(st.U, st.E, st.phi, st.pi, st.step)
    d = g.diagnostics()
    tau = 6 * 0.125
    e = O.energy(n, tau, 1, st.U, st.E, st.phi, st.pi)
    assert abs(d[0] - O.gauss_rel(st)) < 1e-12 * max(1.0, O.gauss_rel(st))
    assert rel_err(d[1:5], e) < 1e-12
    assert d[5] < 1e-13 and d[7] == 0
