"""Batched multi-event runs (uneven lattices, own particle ensembles) against the
oracle, through the C ABI."""
import numpy as np
import pytest

import oracle as O
from gpu_common import rel_err

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_2307_07999_gb300")
W = pytest.importorskip("paper_2307_07999_gb300.workloads")

HBARC = 0.1973269804


def small_events(prec, tol=1e-14, np_=400):
    """Four events with different sizes (one ragged against the 32-wide tiles) and
    step counts; L chosen so that g^2 mu a ~ 1 (well-conditioned tau = 0+ solve)."""
    spec = [(24, 2.4, 1.8), (40, 4.0, 2.2), (32, 2.6, 2.0), (48, 4.2, 1.6)]
    evs, pps = [], []
    for e, (n, L, g2mu) in enumerate(spec):
        s = W.event_seed(9, e)
        gp = W.glasma_params(n, L, g2mu, s, prec, tau_end_fm=0.35, reunit_every=(0 if prec == 0 else 16))
        gp.newton_tol = tol
        evs.append(gp)
        pps.append(W.charm_params(np_, s, mass=1.5, p_max=3.0, tau_form=0.08))
    return evs, pps


def oracle_event(gp, pp, tol, particle_idx=None):
    n = gp.n
    a_fm = gp.L_fm / n
    a = a_fm / HBARC
    st, iters, fails = O.glasma_init(n, gp.n_sheets, gp.g2mu_GeV * a, gp.m_ir_GeV * a, gp.seed, gp.dtau_over_a,
                                     tol=tol)
    P = O.particles_init(pp.n_particles, n, pp.mass_GeV * a, pp.init_kind, pp.p_min_GeV * a, pp.p_max_GeV * a,
                         pp.seed)
    if particle_idx is not None:
        sub = O.Particles(len(particle_idx))
        for k in ("x", "y", "eta", "px", "py", "peta", "Q", "p0"):
            getattr(sub, k)[...] = getattr(P, k)[particle_idx]
        P = sub
    n_form = max(1, int(round(pp.tau_form_fm / (gp.dtau_over_a * a_fm))))
    n_steps = int(np.ceil(gp.tau_end_fm / (gp.dtau_over_a * a_fm) - 1e-9))
    while st.step < n_form:
        st = O.field_step(st, gp.dtau_over_a)
    rows = [(n_form * gp.dtau_over_a * a_fm, 0, 0, 0, P.np)]
    while st.step < n_steps:
        nx = O.field_step(st, gp.dtau_over_a)
        acc = O.push(P, st, nx, gp.dtau_over_a, pp.mass_GeV * a)
        rows.append((nx.step * gp.dtau_over_a * a_fm, *(acc[:3] / acc[3] / a ** 2), acc[3]))
        st = nx
    return np.array(rows), P, st


@pytest.fixture(scope="module")
def fp64_batch():
    evs, pps = small_events(0)
    B = G.Batch(evs, pps)
    assert B.init() == 0
    return B, evs, pps


def test_batch_modes_agree(fp64_batch):
    B, evs, pps = fp64_batch
    tabs = {}
    for mode in ("graph", "eager", "per_event", "persistent", "graph"):
        B.run(mode)
        tabs[mode] = [B.broadening(e) for e in range(len(evs))]
    errs = {m: max(rel_err(tabs[m][e][:, 1:4], tabs["graph"][e][:, 1:4]) for e in range(len(evs)))
            for m in ("eager", "per_event", "persistent")}
    print("mode errors vs graph:", errs)
    for m, v in errs.items():
        assert v < 1e-13, (m, v)


def test_batch_fp64_matches_oracle(fp64_batch):
    B, evs, pps = fp64_batch
    B.run("graph")
    su, ps = B.work()
    assert su == sum(gp.n ** 2 * (int(np.ceil(gp.tau_end_fm / (gp.dtau_over_a * gp.L_fm / gp.n) - 1e-9)) - 1)
                     for gp in evs)
    for e in range(len(evs)):
        want, P, st = oracle_event(evs[e], pps[e], 1e-14)
        got = B.broadening(e)
        assert got.shape == want.shape
        assert np.abs(got[:, 0] - want[:, 0]).max() < 1e-12
        assert rel_err(got[:, 1:4], want[:, 1:4]) < 1e-10, e
        d = B.diagnostics(e)
        assert d[7] == 0 and d[5] < 1e-12
        part = B.get_particles(e)
        assert rel_err(part["px"], P.px) < 1e-10 and rel_err(part["Q"], P.Q) < 1e-10


def test_batch_fp32_matches_oracle():
    evs, pps = small_events(1, tol=1e-14)
    B = G.Batch(evs, pps)
    B.init()
    B.run("graph")
    for e in range(len(evs)):
        want, P, st = oracle_event(evs[e], pps[e], 1e-14)
        got = B.broadening(e)
        e_dp = rel_err(got[:, 1:4], want[:, 1:4])
        e_k = rel_err(G.kappa_qhat(got)[:, 1:], O.kappa_qhat(want)[:, 1:])
        d = B.diagnostics(e)
        print(f"event {e}: dp2 {e_dp:.2e} kappa {e_k:.2e} gauss {d[0]:.2e} unitarity {d[5]:.2e}")
        assert e_dp < 1e-4 and e_k < 1e-4
        assert d[0] < 1e-5


def test_tile_variants_are_bit_identical_and_tuning_picks_one():
    """Every FP32 field tile shape (the lattices include sizes that are ragged against
    each shape) gives the same particle states bit for bit: the per-site arithmetic
    does not depend on the tile.  (The FP64 broadening sums and monitors are atomic
    accumulations whose order varies from run to run: equal to 1e-12.)  The tuner
    times every shape and keeps one."""
    evs, pps = small_events(1, tol=1e-14)
    B = G.Batch(evs, pps)
    B.init()
    nv = G.field_tile_variants(G.GLASMA_FP32)
    assert nv >= 2 and G.field_tile_variants(G.GLASMA_FP64) == 1
    shapes = [G.field_tile_shape(G.GLASMA_FP32, v) for v in range(nv)]
    assert shapes[0] == (32, 4, 3) and len(set(shapes)) == nv
    keys = ("x", "y", "eta", "px", "py", "peta", "Q")
    ref = None
    for v in range(nv):
        B.set_variant(v)
        assert B.variant == v
        for mode in ("eager", "graph"):
            B.run(mode)
            parts = [B.get_particles(e) for e in range(len(evs))]
            tabs = [B.broadening(e) for e in range(len(evs))]
            mons = [B.diagnostics(e) for e in range(len(evs))]
            if ref is None:
                ref = (parts, tabs, mons)
            for e in range(len(evs)):
                for k in keys:
                    assert np.array_equal(parts[e][k], ref[0][e][k]), (shapes[v], mode, e, k)
                assert rel_err(tabs[e], ref[1][e]) < 1e-12, (shapes[v], mode, e)
                assert rel_err(mons[e][:6], ref[2][e][:6]) < 1e-12, (shapes[v], mode, e)
    # the push kernels (fields through L1, or staged in shared memory): the same source
    # compiled into two kernels, whose FMA contractions may differ: equal to FP32 rounding
    # (the record push, variant 2, contracts the same pieces in another order: its FP32
    # results are checked against the oracle in test_gpu_records.py)
    B.set_variant(0)
    assert G.lib().glasma_push_variants() == 4
    for pv in range(2):
        B.set_push_variant(pv)
        assert B.push_variant == pv
        B.run("graph")
        for e in range(len(evs)):
            part = B.get_particles(e)
            for k in keys:
                assert rel_err(part[k], ref[0][e][k]) < 2e-6, (pv, e, k, rel_err(part[k], ref[0][e][k]))
    chosen, ms = B.tune(steps=4)
    print("tile variant times (ms):", {shapes[v]: round(ms[v], 3) for v in range(nv)}, "chosen", shapes[chosen],
          "push kernel", B.push_variant)
    assert 0 <= chosen < nv and B.variant == chosen and all(m > 0 for m in ms)
    assert B.push_variant in (0, 1, 2, 3)
    B.run("graph")
    tol = 2e-6 if B.push_variant in (0, 1) else 1e-4
    assert rel_err(B.get_particles(0)["px"], ref[0][0]["px"]) < tol


def test_full_size_batch_sampled():
    """The benchmarked workload at full size, in the launch configuration bench.py times
    (graph mode, FP32): monitors of all 64 events, and event 0 (128^2, 10k charm)
    checked on a sample of 200 particles that the FP64 oracle pushes one by one through
    its own evolution of the same event."""
    evs, pps = W.batched_uneven()
    B = G.Batch(evs, pps)
    fails = B.init()
    assert fails == 0
    B.tune(steps=4)  # the tile shape bench.py runs with
    B.run("graph")
    for e in range(len(evs)):
        d = B.diagnostics(e)
        assert d[7] == 0, e
        assert d[0] < 1e-5, (e, d[0])
        assert d[5] < 1e-5, (e, d[5])
        tab = B.broadening(e)
        assert np.all(np.isfinite(tab)) and np.all(tab[1:, 4] == pps[e].n_particles)
    idx = np.random.default_rng(0).choice(pps[0].n_particles, 200, replace=False)
    want, P, st = oracle_event(evs[0], pps[0], evs[0].newton_tol, particle_idx=idx)
    got = B.get_particles(0)
    a = evs[0].L_fm / evs[0].n / HBARC
    p_got = np.stack([got["px"][idx], got["py"][idx]], 1)
    p_want = np.stack([P.px, P.py], 1)
    dp_got = ((p_got ** 2).sum(1) - (P.p0[:, :2] ** 2).sum(1)).mean()
    dp_want = ((p_want ** 2).sum(1) - (P.p0[:, :2] ** 2).sum(1)).mean()
    rel = np.abs(p_got - p_want).max(1) / np.maximum(np.abs(p_want).max(1), 1e-3 / a)
    print(f"sampled particles: median rel {np.median(rel):.2e}, 95% {np.quantile(rel, 0.95):.2e}, "
          f"<dp_T^2> rel {abs(dp_got - dp_want) / abs(dp_want):.2e}")
    assert np.quantile(rel, 0.9) < 1e-3
    assert abs(dp_got - dp_want) < 1e-3 * abs(dp_want)
    # the largest event (512^2, 409 batched FP32 steps) against the oracle's own FP64
    # evolution of it: the four energy densities of the final state (global observables,
    # insensitive to the chaotic growth of local rounding differences) within 1e-4
    big = max(range(len(evs)), key=lambda e: (evs[e].n, -e))
    gp = evs[big]
    a = gp.L_fm / gp.n / HBARC
    st, _, fails_o = O.glasma_init(gp.n, gp.n_sheets, gp.g2mu_GeV * a, gp.m_ir_GeV * a, gp.seed, gp.dtau_over_a,
                                   tol=gp.newton_tol)
    n_steps = int(np.ceil(gp.tau_end_fm / (gp.dtau_over_a * gp.L_fm / gp.n) - 1e-9))
    while st.step < n_steps:
        st = O.field_step(st, gp.dtau_over_a)
    want_e = O.energy(gp.n, st.step * gp.dtau_over_a, 1, st.U, st.E, st.phi, st.pi)
    d = B.diagnostics(big)
    print(f"event {big} ({gp.n}^2): energies {d[1:5]} vs oracle {want_e}")
    assert rel_err(d[1:5], want_e) < 1e-4, (d[1:5], want_e)
    assert abs(d[6] - st.step * gp.dtau_over_a) < 1e-9


def test_batch_import_from_device_memory(fp64_batch):
    """The batch's initial state imported from a device buffer (a caller's staging copy)
    gives the run of the state imported from host memory."""
    import torch

    B, evs, pps = fp64_batch
    nb = B.state_bytes()
    host = torch.empty(nb, dtype=torch.uint8, pin_memory=True)
    B.export_state(host)
    B.import_state(host)
    B.run("graph")
    want = [B.broadening(e) for e in range(len(evs))]
    staged = host.to("cuda")
    torch.cuda.synchronize()
    B.import_state(staged)
    B.run("graph")
    for e in range(len(evs)):
        got = B.broadening(e)
        assert rel_err(got[:, 1:4], want[e][:, 1:4]) < 1e-13, e


def test_graph_timing_nodes(fp64_batch):
    """Event-record nodes around the field launches of the captured graph: one pair per
    iteration of the run, durations that fit in the span, and the same results."""
    B, evs, pps = fp64_batch
    B.run("graph")
    want = [B.broadening(e) for e in range(len(evs))]
    B.set_graph_timing(True)
    B.run("graph")
    field_ms, n, span = B.graph_times()
    n_iter = max(int(np.ceil(gp.tau_end_fm / (gp.dtau_over_a * gp.L_fm / gp.n) - 1e-9)) for gp in evs) - 1
    assert n == n_iter and 0 < field_ms <= span
    for e in range(len(evs)):
        assert rel_err(B.broadening(e)[:, 1:4], want[e][:, 1:4]) < 1e-13
    B.set_graph_timing(False)
    B.run("graph")
    with pytest.raises(G.GlasmaError):
        B.graph_times()


def test_push_stream_gives_the_same_run(fp64_batch):
    """Pushes on a second stream (push k after field k, field k+2 after push k): the same
    particles bit for bit and the same broadening tables, in graph and eager modes."""
    B, evs, pps = fp64_batch
    B.run("graph")
    want = [(B.broadening(e), B.get_particles(e)) for e in range(len(evs))]
    B.set_push_stream(True)
    for mode in ("graph", "eager", "graph"):
        B.run(mode)
        for e in range(len(evs)):
            tab, part = B.broadening(e), B.get_particles(e)
            assert rel_err(tab[:, 1:4], want[e][0][:, 1:4]) < 1e-13, (mode, e)
            for k in part:
                assert np.array_equal(part[k], want[e][1][k]), (mode, e, k)
    B.set_push_stream(False)
