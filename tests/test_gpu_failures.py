"""Failure detection without a GPU fault: non-finite fields injected on the host are
reported as GLASMA_ERR_NONFINITE, and the persistent mode's bounded grid-barrier wait,
made to run out on purpose, ends the launch and is reported as GLASMA_ERR_TIMEOUT; in
both cases the same context or batch is used again afterwards and gives correct
results."""
import ctypes as C

import numpy as np
import pytest

from gpu_common import random_state, rel_err
from test_gpu_batch import small_events

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_2307_07999_gb300")
L = pytest.importorskip("paper_2307_07999_gb300._lib")

NONFINITE, TIMEOUT = -3, -4


def _diag_status(g):
    out = np.zeros(8)
    st = L.lib().glasma_diagnostics(g.handle, out.ctypes.data_as(C.c_void_p))
    return st, out


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("where", ["E", "pi", "U"])
def test_injected_nan_is_reported_and_the_context_recovers(prec, where):
    n = 12
    st = random_state(n, 21)
    g = G.Glasma(n, 2.0, precision=prec, tau_end_fm=10.0)
    g.set_state(st.U, st.E, st.phi, st.pi, 3)
    s0, d0 = _diag_status(g)
    assert s0 == 0 and d0[7] == 0
    bad = st.copy()
    if where == "E":
        bad.E[17, 1, 4] = np.nan
    elif where == "pi":
        bad.pi[5, 2] = np.inf
    else:
        bad.U[40, 0, 1, 2] = complex(np.nan, 0.0)
    g.set_state(bad.U, bad.E, bad.phi, bad.pi, 3)
    s1, d1 = _diag_status(g)
    assert s1 == NONFINITE and d1[7] > 0
    assert L.lib().glasma_last_error()
    # one step spreads it to the neighbours; still reported, no fault
    g.step(1)
    s2, d2 = _diag_status(g)
    assert s2 == NONFINITE and d2[7] >= d1[7]
    # the same context takes a clean state again
    g.set_state(st.U, st.E, st.phi, st.pi, 3)
    s3, d3 = _diag_status(g)
    assert s3 == 0 and d3[7] == 0
    assert d3[:6] == pytest.approx(d0[:6], rel=1e-12, abs=1e-15)


def test_persistent_barrier_timeout_is_reported_and_the_batch_recovers():
    evs, pps = small_events(0, np_=200)
    B = G.Batch(evs, pps)
    assert B.init() == 0
    B.run("graph")
    ref = [B.broadening(e) for e in range(len(evs))]
    # a bound of one poll: the first CTAs at a barrier give up before the others arrive
    B.set_wait_limit(1)
    B.run("persistent")
    with pytest.raises(G.GlasmaError) as ei:
        B.broadening(0)
    assert ei.value.status == TIMEOUT
    # reported once: the error word is cleared when read
    B.broadening(0)
    # back to the default bound: the same batch runs to the end and agrees with the graph run
    B.set_wait_limit(0)
    B.run("persistent")
    for e in range(len(evs)):
        assert rel_err(B.broadening(e)[:, 1:4], ref[e][:, 1:4]) < 1e-13
    B.run("graph")
    for e in range(len(evs)):
        assert rel_err(B.broadening(e)[:, 1:4], ref[e][:, 1:4]) == 0.0


def test_wait_limit_arguments_are_checked():
    evs, pps = small_events(0, np_=10)
    B = G.Batch(evs[:1], pps[:1])
    with pytest.raises(G.GlasmaError):
        B.set_wait_limit(-1)
    with pytest.raises(G.GlasmaError):
        B.set_wait_limit(1 << 41)
