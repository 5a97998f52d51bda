"""The benchmarked workload at full size, in the launch configuration bench.py times: the
64-event batch (16 each of 128^2, 256^2, 384^2, 512^2, 10k charm per event, FP32 fields
and particles, FP64 accumulators), tuned as bench.py tunes it and run in graph mode.
One whole 128^2 event and one whole 256^2 event (every one of their 10k quarks, every
step) are compared with the oracle's own FP64 evolution of the same events (its own
initial conditions from the same seeds): the complete broadening tables <dp_i^2>(tau)
and the Eq. 3 coefficients."""
import numpy as np
import pytest

import oracle as O
from gpu_common import rel_err
from test_gpu_batch import oracle_event

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_2307_07999_gb300")
W = pytest.importorskip("paper_2307_07999_gb300.workloads")

DP2_TOL = 1e-4     # <dp_i^2>(tau), relative to the table's largest value
KAPPA_TOL = 1e-4   # d<dp_i^2>/dtau, relative to its largest value (kappa crosses zero)


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
    assert evs[event].n == (128 if event == 0 else 256)
    want, P, st = oracle_event(evs[event], pps[event], evs[event].newton_tol)
    got = B.broadening(event)
    assert got.shape == want.shape
    assert np.abs(got[:, 0] - want[:, 0]).max() < 1e-9
    assert np.all(got[:, 4] == want[:, 4])
    e_dp = rel_err(got[:, 1:4], want[:, 1:4])
    tg, tw = G.broadening_transport(got), O.transport_coefficients(want)
    e_k = rel_err(tg[:, 1:4], tw[:, 1:4])
    e_kl = rel_err(tg[:, 4:7], tw[:, 4:7])
    e_an = rel_err(tg[1:, 7], tw[1:, 7])
    print(f"event {event} ({evs[event].n}^2, push kernel {B.push_variant}): <dp^2> {e_dp:.2e}, "
          f"d<dp_i^2>/dtau {e_k:.2e}, kappa_T/kappa_L/total {e_kl:.2e}, anisotropy {e_an:.2e}")
    assert e_dp < DP2_TOL
    assert e_k < KAPPA_TOL and e_kl < KAPPA_TOL
    assert e_an < DP2_TOL
    d = B.diagnostics(event)
    assert d[0] < 1e-5 and d[7] == 0
