"""Lattice-correlator estimators (Sec. 2, Eqs. 4 and 5) through the C ABI against the
FP64 oracle on the same initial state: FP64 to 1e-10, FP32 to 1e-4."""
import numpy as np
import pytest

import oracle as O
from gpu_common import lattice_units, rel_err

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_2307_07999_gb300")

HBARC = 0.1973269804


def oracle_run(n, L, seed, tau_start, ox0, n_steps):
    a_fm, a, g2mua, mira = lattice_units(n, L)
    st, iters, fails = O.glasma_init(n, 10, g2mua, mira, seed, 0.125)
    st0 = st.copy()
    first = max(1, int(round(tau_start / (0.125 * a_fm))))
    while st.step < first:
        st = O.field_step(st, 0.125)
    C = O.Correlators(n, ox0=ox0)
    rows = [(first * 0.125 * a_fm, 0, 0, 0, 0, 0, 0)]
    while st.step < n_steps:
        nx = O.field_step(st, 0.125)
        out = C.step(st, nx, 0.125)
        rows.append((nx.step * 0.125 * a_fm, *(out / a ** 2)))
        st = nx
    return st0, np.array(rows), first


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-4)])
def test_correlators_match_oracle(prec, tol):
    n, L, seed, tau_start, ox0, n_steps = 16, 3.2, 77, 0.05, 0.3, 45
    st0, want, first = oracle_run(n, L, seed, tau_start, ox0, n_steps)
    g = G.Glasma(n, L, precision=prec, tau_end_fm=2.0, seed=seed, reunit_every=(0 if prec == 0 else 16))
    g.set_state(st0.U, st0.E, st0.phi, st0.pi, 1)
    g.step(first - 1)
    c = G.Correlators(g, tau_start_fm=tau_start, ox0=ox0)
    g.step(n_steps - first)
    got = c.table()
    assert got.shape == want.shape
    assert np.abs(got[:, 0] - want[:, 0]).max() < 1e-12
    for k in range(1, 7):
        e = rel_err(got[:, k], want[:, k])
        assert e < tol, (k, e)
    # the lightlike paths crossed cell faces (the Wilson lines are exercised)
    assert np.floor(ox0 + (n_steps - first) * 0.125) >= 4


def test_correlators_advance_once_per_step_with_particles():
    """Attached to a context that a particle push advances: one accumulation per step."""
    n, L, seed = 12, 2.4, 5
    st0, want, first = oracle_run(n, L, seed, 0.0, 0.5, 20)
    g = G.Glasma(n, L, precision=0, tau_end_fm=2.0, seed=seed)
    g.set_state(st0.U, st0.E, st0.phi, st0.pi, 1)
    c = G.Correlators(g, tau_start_fm=0.0, ox0=0.5)
    p = G.CPIC(g, 50, 1.5, 0.0, p_max_GeV=1.0, seed=3)
    p.init()
    p.push(19)
    got = c.table()
    assert got.shape == want.shape
    assert rel_err(got[:, 1:], want[:, 1:]) < 1e-10
