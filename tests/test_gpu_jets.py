"""Jets (light-like massless partons along +x, q^ from the transverse broadening;
Sec. 2 of arXiv:2307.07999), through the batch C ABI.  The parton momenta
{2, 5, 10} GeV of one Glasma event are three ensembles of three batch events with the
same field seed: the fields of the three evolve bit for bit alike."""
import numpy as np
import pytest

import oracle as O
from gpu_common import rel_err

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_2307_07999_gb300")
W = pytest.importorskip("paper_2307_07999_gb300.workloads")

HBARC = 0.1973269804
P_JET = (2.0, 5.0, 10.0)


def jet_events(n, L, tau_end, n_partons, prec, field_seeds, tau_form=0.3, tol=1e-12):
    evs, pps = [], []
    for fs in field_seeds:
        for k, p in enumerate(P_JET):
            gp = W.glasma_params(n, L, 2.0, fs, prec, tau_end_fm=tau_end, reunit_every=(0 if prec == 0 else 16))
            gp.newton_tol = tol
            pp = W.charm_params(n_partons, fs + 7919 * (k + 1), mass=0.0, p_max=p, tau_form=tau_form)
            pp.init_kind, pp.p_min_GeV = 1, p
            evs.append(gp)
            pps.append(pp)
    return evs, pps


def oracle_jets(gp, pp, tol):
    n = gp.n
    a_fm = gp.L_fm / n
    a = a_fm / HBARC
    st, iters, fails = O.glasma_init(n, gp.n_sheets, gp.g2mu_GeV * a, gp.m_ir_GeV * a, gp.seed, gp.dtau_over_a,
                                     tol=tol)
    P = O.particles_init(pp.n_particles, n, 0.0, 1, pp.p_min_GeV * a, pp.p_max_GeV * a, pp.seed)
    n_form = max(1, int(round(pp.tau_form_fm / (gp.dtau_over_a * a_fm))))
    n_steps = int(np.ceil(gp.tau_end_fm / (gp.dtau_over_a * a_fm) - 1e-9))
    while st.step < n_form:
        st = O.field_step(st, gp.dtau_over_a)
    rows = [(n_form * gp.dtau_over_a * a_fm, 0, 0, 0, P.np)]
    while st.step < n_steps:
        nx = O.field_step(st, gp.dtau_over_a)
        acc = O.push(P, st, nx, gp.dtau_over_a, 0.0)
        rows.append((nx.step * gp.dtau_over_a * a_fm, *(acc[:3] / acc[3] / a ** 2), acc[3]))
        st = nx
    return np.array(rows), P


@pytest.mark.parametrize("prec", [0, 1])
def test_jets_small_vs_oracle(prec):
    """32^2, L = 3.2 fm (g^2 mu a ~ 1), partons formed at 0.3 fm/c and followed to
    0.6 fm/c: FP64 to 1e-10; FP32 <dp^2> and q^ to 1e-4 of their largest values."""
    evs, pps = jet_events(32, 3.2, 0.6, 300, prec, [W.event_seed(4, 0)], tol=1e-14)
    B = G.Batch(evs, pps)
    assert B.init() == 0
    B.run("graph")
    for e in range(3):
        want, P = oracle_jets(evs[e], pps[e], 1e-14)
        got = B.broadening(e)
        assert got.shape == want.shape
        if prec == 0:
            assert rel_err(got[:, 1:4], want[:, 1:4]) < 1e-10, e
            part = B.get_particles(e)
            assert rel_err(part["px"], P.px) < 1e-10 and rel_err(part["Q"], P.Q) < 1e-10
        else:
            assert rel_err(got[:, 1:4], want[:, 1:4]) < 1e-4, e
            q_got, q_want = G.kappa_qhat(got), O.kappa_qhat(want)
            assert rel_err(q_got[:, 2:], q_want[:, 2:]) < 1e-4, e  # q^_y, q^_z
    # the three ensembles saw the same fields: same monitors
    d = [B.diagnostics(e) for e in range(3)]
    assert d[0][:6] == pytest.approx(d[1][:6], rel=1e-12) and d[0][:6] == pytest.approx(d[2][:6], rel=1e-12)


def test_jets_full_size_properties():
    """The jets configuration at full size: 1024^2, L = 10 fm, 1M massless partons per
    event at each of 2, 5 and 10 GeV, formed at 0.3 fm/c, to 1 fm/c (820 steps); one
    field event (three ensembles).  Checked by what holds at any size: Gauss law and
    unitarity of every event, every parton pushed at every step, the colour charges on
    their Casimir surface, finite broadening."""
    evs, pps = jet_events(1024, 10.0, 1.0, 1 << 20, 1, [W.event_seed(4, 1)])
    B = G.Batch(evs, pps)
    assert B.init() == 0
    B.tune(steps=4)
    B.run("graph")
    for e in range(len(evs)):
        d = B.diagnostics(e)
        assert d[7] == 0 and d[0] < 1e-5 and d[5] < 1e-5, (e, d)
        tab = B.broadening(e)
        assert np.all(np.isfinite(tab)) and np.all(tab[1:, 4] == pps[e].n_particles)
        assert np.all(tab[1:, 2:4] > 0)
        part = B.get_particles(e)
        idx = np.random.default_rng(e).choice(pps[e].n_particles, 20000, replace=False)
        Q = part["Q"][idx]
        q2 = (Q ** 2).sum(1)
        assert np.abs(q2 - 4.0).max() < 1e-3, np.abs(q2 - 4.0).max()
    # q^_y, q^_z of the three momenta: finite and of one scale
    q = np.array([G.kappa_qhat(B.broadening(e))[:, 2:].mean(0) for e in range(len(evs))])
    print("mean q^_y, q^_z (GeV^2/fm) at p = 2, 5, 10 GeV:", q.tolist())
    assert np.all(np.isfinite(q))
