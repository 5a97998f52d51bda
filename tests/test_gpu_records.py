"""The record push (batched push variant 2; the split push, variant 3, is checked here too):
the batched field launch writes, for every
cell a particle occupies, the pieces of the site-centred fields it computes anyway
(time-centred E and pi, phi, the phi transports, three clover leaves, and the neighbour
pieces of the cells +x, +y), and the push reads that one record instead of gathering 35
field groups.  Checked against the oracle (FP64 1e-10, FP32 1e-4), for both momentum
kicks, and shown to leave the field evolution untouched."""
import numpy as np
import pytest

import oracle as O
from gpu_common import rel_err
from test_gpu_batch import HBARC, oracle_event, small_events

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_2307_07999_gb300")
W = pytest.importorskip("paper_2307_07999_gb300.workloads")

RECORD = 2
SPLIT = 3   # the split push: force kernel (gather) + move kernel


def oracle_event_int(gp, pp, tol, integrator):
    """oracle_event with the momentum kick of the given integrator"""
    if integrator == 0:
        return oracle_event(gp, pp, tol)
    n = gp.n
    a_fm = gp.L_fm / n
    a = a_fm / HBARC
    st, _, _ = O.glasma_init(n, gp.n_sheets, gp.g2mu_GeV * a, gp.m_ir_GeV * a, gp.seed, gp.dtau_over_a, tol=tol)
    P = O.particles_init(pp.n_particles, n, pp.mass_GeV * a, pp.init_kind, pp.p_min_GeV * a, pp.p_max_GeV * a,
                         pp.seed)
    n_form = max(1, int(round(pp.tau_form_fm / (gp.dtau_over_a * a_fm))))
    n_steps = int(np.ceil(gp.tau_end_fm / (gp.dtau_over_a * a_fm) - 1e-9))
    while st.step < n_form:
        st = O.field_step(st, gp.dtau_over_a)
    rows = [(n_form * gp.dtau_over_a * a_fm, 0, 0, 0, P.np)]
    while st.step < n_steps:
        nx = O.field_step(st, gp.dtau_over_a)
        acc = O.push(P, st, nx, gp.dtau_over_a, pp.mass_GeV * a, integrator=integrator)
        rows.append((nx.step * gp.dtau_over_a * a_fm, *(acc[:3] / acc[3] / a ** 2), acc[3]))
        st = nx
    return np.array(rows), P, st


@pytest.mark.parametrize("pv", [RECORD, SPLIT])
@pytest.mark.parametrize("integrator", [0, 1])
def test_record_push_fp64_matches_oracle(integrator, pv):
    evs, pps = small_events(0)
    for pp in pps:
        pp.integrator = integrator
    B = G.Batch(evs, pps)
    assert B.init() == 0
    B.set_push_variant(pv)
    assert B.push_variant == pv
    for mode in ("graph", "eager"):
        B.run(mode)
        for e in range(len(evs)):
            want, P, st = oracle_event_int(evs[e], pps[e], 1e-14, integrator)
            got = B.broadening(e)
            assert got.shape == want.shape
            assert rel_err(got[:, 1:4], want[:, 1:4]) < 1e-10, (mode, e)
            assert rel_err(G.kappa_qhat(got)[:, 1:], O.kappa_qhat(want)[:, 1:]) < 1e-10, (mode, e)
            part = B.get_particles(e)
            for k in ("px", "py", "peta", "eta", "Q"):
                assert rel_err(part[k], getattr(P, k)) < 1e-10, (mode, e, k)
            n = evs[e].n
            for k, w in (("x", P.x), ("y", P.y)):
                d = np.abs(part[k] - w)
                assert np.minimum(d, n - d).max() < 1e-10, (mode, e, k)


@pytest.mark.parametrize("pv", [RECORD, SPLIT])
def test_record_push_fp32_matches_oracle(pv):
    evs, pps = small_events(1, tol=1e-14)
    B = G.Batch(evs, pps)
    B.init()
    B.set_push_variant(pv)
    B.run("graph")
    for e in range(len(evs)):
        want, P, st = oracle_event(evs[e], pps[e], 1e-14)
        got = B.broadening(e)
        e_dp = rel_err(got[:, 1:4], want[:, 1:4])
        e_k = rel_err(G.kappa_qhat(got)[:, 1:], O.kappa_qhat(want)[:, 1:])
        print(f"event {e}: record push FP32 dp2 {e_dp:.2e} kappa {e_k:.2e}")
        assert e_dp < 1e-4 and e_k < 1e-4


@pytest.mark.parametrize("prec", [0, 1])
def test_records_leave_the_fields_unchanged(prec):
    """The field launches that write records run the field arithmetic of the plain ones:
    the final fields of every event agree (FP64: monitors to their FP64 summation order;
    FP32: to the growth of rounding differences, since the compiler may contract some
    multiply-adds of the two kernels differently), and eager and graph runs of the record
    push agree bit for bit."""
    evs, pps = small_events(prec, tol=1e-14)
    B = G.Batch(evs, pps)
    B.init()
    B.set_push_variant(0)
    B.run("graph")
    mon0 = [B.diagnostics(e) for e in range(len(evs))]
    B.set_push_variant(RECORD)
    B.run("graph")
    mon1 = [B.diagnostics(e) for e in range(len(evs))]
    parts_g = [B.get_particles(e) for e in range(len(evs))]
    tol = 1e-12 if prec == 0 else 1e-5
    for e in range(len(evs)):
        assert rel_err(mon1[e][:6], mon0[e][:6]) < tol, e
    B.run("eager")
    for e in range(len(evs)):
        part = B.get_particles(e)
        for k in part:
            assert np.array_equal(part[k], parts_g[e][k]), (e, k)


def test_record_push_with_empty_and_crowded_events():
    """An event without particles next to an event with several particles in most cells."""
    evs, pps = small_events(0)
    pps[1].n_particles = 0
    pps[0].n_particles = 3000  # 24^2 = 576 cells
    B = G.Batch(evs[:2], pps[:2])
    assert B.init() == 0
    B.set_push_variant(RECORD)
    B.run("graph")
    want, P, st = oracle_event(evs[0], pps[0], 1e-14)
    assert rel_err(B.broadening(0)[:, 1:4], want[:, 1:4]) < 1e-10
    t1 = B.broadening(1)
    assert np.all(t1[:, 1:4] == 0)


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-4)])
def test_record_push_on_the_smallest_lattices(prec, tol):
    """Lattices of 2 and 3 sites per side: the neighbour cells +x and -x (and +y, -y) of a
    cell coincide or wrap at once, so one site writes several neighbour pieces of the same
    record; a 5^2 lattice ragged against every tile shape beside them."""
    evs, pps = [], []
    for e, (n, L) in enumerate([(2, 0.2), (3, 0.3), (5, 0.5)]):  # a = 0.1 fm: g^2 mu a ~ 1
        s = W.event_seed(9, 40 + e)
        gp = W.glasma_params(n, L, 2.0, s, prec, tau_end_fm=0.08, reunit_every=(0 if prec == 0 else 16))
        gp.newton_tol = 1e-14
        evs.append(gp)
        pps.append(W.charm_params(50, s, mass=1.5, p_max=3.0, tau_form=0.01))
    B = G.Batch(evs, pps)
    assert B.init() == 0
    B.set_push_variant(RECORD)
    B.run("graph")
    for e in range(len(evs)):
        want, P, st = oracle_event(evs[e], pps[e], 1e-14)
        got = B.broadening(e)
        assert got.shape == want.shape
        assert rel_err(got[:, 1:4], want[:, 1:4]) < tol, e
