"""The benchmarked workload at full size, in the launch configuration bench.py times: the
64-event batch (16 each of 128^2, 256^2, 384^2, 512^2, 10k charm per event, FP32 fields
and particles, FP64 accumulators), tuned as bench.py tunes it and run in graph mode.
One whole 128^2 event and one whole 256^2 event (every one of their 10k quarks, every
step) are compared with the oracle's own FP64 evolution of the same events (its own
initial conditions from the same seeds): the complete broadening tables <dp_i^2>(tau),
the Eq. 3 coefficients kappa_T, kappa_L and the anisotropy.

Tolerances: <dp_i^2> and the anisotropy within 1e-4 of their largest values.  kappa
within 1e-4, or within twice the error that FP32 storage of the fields alone causes,
whichever is larger: the nearest-grid-point gather makes a quark's force jump when a
rounding-level change moves one of its cell crossings by a step, and kappa, a one-step
difference of <dp^2>, shows each such jump.  The oracle measures that floor itself: the
same FP64 evolution with every stored field rounded to FP32 after each step."""
import numpy as np
import pytest

import oracle as O
from gpu_common import rel_err
from test_gpu_batch import HBARC, oracle_event

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_2307_07999_gb300")
W = pytest.importorskip("paper_2307_07999_gb300.workloads")

DP2_TOL = 1e-4     # <dp_i^2>(tau) and the anisotropy, relative to their largest values
KAPPA_TOL = 1e-4   # d<dp_i^2>/dtau, relative to its largest value (kappa crosses zero)


def _round_fp32(st):
    """the state with every stored real rounded to FP32 (the oracle stays FP64 otherwise)"""
    st.U.real[...] = st.U.real.astype(np.float32)
    st.U.imag[...] = st.U.imag.astype(np.float32)
    for k in ("E", "phi", "pi"):
        a = getattr(st, k)
        a[...] = a.astype(np.float32)
    return st


def oracle_event_fp32_storage(gp, pp, tol):
    """oracle_event with the fields rounded to FP32 after every step (pushes in FP64)"""
    n = gp.n
    a_fm = gp.L_fm / n
    a = a_fm / HBARC
    st, _, _ = O.glasma_init(n, gp.n_sheets, gp.g2mu_GeV * a, gp.m_ir_GeV * a, gp.seed, gp.dtau_over_a, tol=tol)
    st = _round_fp32(st)
    P = O.particles_init(pp.n_particles, n, pp.mass_GeV * a, pp.init_kind, pp.p_min_GeV * a, pp.p_max_GeV * a,
                         pp.seed)
    n_form = max(1, int(round(pp.tau_form_fm / (gp.dtau_over_a * a_fm))))
    n_steps = int(np.ceil(gp.tau_end_fm / (gp.dtau_over_a * a_fm) - 1e-9))
    while st.step < n_form:
        st = _round_fp32(O.field_step(st, gp.dtau_over_a))
    rows = [(n_form * gp.dtau_over_a * a_fm, 0, 0, 0, P.np)]
    while st.step < n_steps:
        nx = _round_fp32(O.field_step(st, gp.dtau_over_a))
        acc = O.push(P, st, nx, gp.dtau_over_a, pp.mass_GeV * a)
        rows.append((nx.step * gp.dtau_over_a * a_fm, *(acc[:3] / acc[3] / a ** 2), acc[3]))
        st = nx
    return np.array(rows)


@pytest.fixture(scope="module")
def headline():
    evs, pps = W.batched_uneven()
    B = G.Batch(evs, pps)
    assert B.init() == 0
    B.tune(steps=8)  # as bench.py: field tile shape and push kernel by measurement
    B.run("graph")
    return B, evs, pps


@pytest.mark.parametrize("event", [0, 16])  # the first 128^2 and the first 256^2 event
def test_headline_events_match_oracle(headline, event):
    B, evs, pps = headline
    gp, pp = evs[event], pps[event]
    assert gp.n == (128 if event == 0 else 256) and pp.n_particles == 10000
    want, P, st = oracle_event(gp, pp, gp.newton_tol)
    got = B.broadening(event)
    assert got.shape == want.shape
    assert np.abs(got[:, 0] - want[:, 0]).max() < 1e-9
    assert np.all(got[:, 4] == want[:, 4])
    tg, tw = G.broadening_transport(got), O.transport_coefficients(want)
    e_dp = rel_err(got[:, 1:4], want[:, 1:4])
    e_k = rel_err(tg[:, 4:6], tw[:, 4:6])     # kappa_T, kappa_L (Eq. 3)
    e_an = rel_err(tg[1:, 7], tw[1:, 7])      # <dp_L^2> / <dp_T^2>
    # the floor FP32 field storage sets on kappa (oracle only)
    t32 = oracle_event_fp32_storage(gp, pp, gp.newton_tol)
    floor = rel_err(O.transport_coefficients(t32)[:, 4:6], tw[:, 4:6])
    print(f"event {event} ({gp.n}^2, push kernel {B.push_variant}): <dp^2> {e_dp:.2e}, "
          f"kappa_T/kappa_L {e_k:.2e} (FP32-storage floor {floor:.2e}), anisotropy {e_an:.2e}")
    assert e_dp < DP2_TOL
    assert e_an < DP2_TOL
    assert e_k < max(KAPPA_TOL, 2.0 * floor)
    d = B.diagnostics(event)
    assert d[0] < 1e-5 and d[7] == 0
