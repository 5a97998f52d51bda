"""The push options beyond the default on the GPU, against the oracle's push with the same
options, through the C ABI (FP64 1e-10 as every push):
- sub-cycled particle steps (cpic_params.substeps = s: s particle steps of dtau/s inside
  one field step, each gathering the step's fields at the particle's current cell);
- the cloud-in-cell gather (cpic_params.interp = 1: the fields of the four sites around
  the particle carried to its cell's site, bilinear weights)."""
import numpy as np
import pytest

import oracle as O
from gpu_common import HBARC, random_particles, random_state, rel_err

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_2307_07999_gb300")
W = pytest.importorskip("paper_2307_07999_gb300.workloads")


def run_pair(n, np_, steps, prec, seed, s, integrator, expanding=1, mass=0.5, interp=0):
    st = random_state(n, seed=seed, step=4)
    P = random_particles(np_, n, seed + 1, mass=mass)
    g = G.Glasma(n, 6.0, precision=prec, expanding=expanding, tau_end_fm=100.0)
    g.set_state(st.U, st.E, st.phi, st.pi, st.step)
    a_gev = (6.0 / n) / HBARC
    c = G.CPIC(g, np_, mass / a_gev, 0.0, integrator=integrator, substeps=s, interp=interp)
    c.set_particles(P.x, P.y, P.eta, P.px, P.py, P.peta, P.Q, P.p0)
    accs = []
    for _ in range(steps):
        nx = O.field_step(st, 0.125, expanding)
        accs.append(O.push(P, st, nx, 0.125, mass, expanding, integrator, s, interp))
        st = nx
    c.push(steps)
    return c, P, np.array(accs), a_gev


@pytest.mark.parametrize("n,s,interp", [(12, 3, 0), (37, 4, 0), (12, 1, 1), (37, 2, 1)])
@pytest.mark.parametrize("integrator", [0, 1])
@pytest.mark.parametrize("expanding", [1, 0])
def test_substeps_and_cic_fp64(n, s, interp, integrator, expanding):
    c, P, accs, a_gev = run_pair(n, 400, 10, 0, 91 + n, s, integrator, expanding, interp=interp)
    got = c.get_particles()
    dx = np.abs(got["x"] - P.x)
    dy = np.abs(got["y"] - P.y)
    assert np.minimum(dx, n - dx).max() < 1e-10 and np.minimum(dy, n - dy).max() < 1e-10
    for k in ("px", "py", "peta", "eta"):
        assert rel_err(got[k], getattr(P, k)) < 1e-10, k
    assert rel_err(got["Q"], P.Q) < 1e-10
    tab = c.broadening()
    assert rel_err(tab[1:, 1:4], accs[:, :3] / accs[:, 3:4] / a_gev ** 2) < 1e-10


@pytest.mark.parametrize("s,interp", [(3, 0), (1, 1)])
def test_substeps_and_cic_fp32(s, interp):
    n = 37
    c, P, accs, a_gev = run_pair(n, 400, 10, 1, 97, s, 1, interp=interp)
    got = c.get_particles()
    assert rel_err(got["px"], P.px) < 2e-5 and rel_err(got["Q"], P.Q) < 2e-5
    tab = c.broadening()
    assert rel_err(tab[1:, 1:4], accs[:, :3] / accs[:, 3:4] / a_gev ** 2) < 1e-4


def test_substeps_batch():
    """A three-event FP64 batch with special ensembles (explicit, s = 3; Boris, s = 2;
    Boris with the cloud-in-cell gather): graph, eager and per-event modes agree to 1e-13
    and with the oracle to 1e-10; the persistent mode refuses it."""
    spec = [(24, 2.4, 1.8, 0, 3, 0), (32, 2.6, 2.0, 1, 2, 0), (28, 2.5, 1.9, 1, 1, 1)]
    evs, pps = [], []
    for e, (n, L, g2mu, integ, s, interp) in enumerate(spec):
        seed = W.event_seed(9, 20 + e)
        gp = W.glasma_params(n, L, g2mu, seed, 0, tau_end_fm=0.3, reunit_every=0)
        gp.newton_tol = 1e-14
        evs.append(gp)
        pp = W.charm_params(300, seed, mass=1.5, p_max=3.0, tau_form=0.08, integrator=integ)
        pp.substeps = s
        pp.interp = interp
        pps.append(pp)
    B = G.Batch(evs, pps)
    assert B.init() == 0
    tabs = {}
    for mode in ("graph", "eager", "per_event"):
        B.run(mode)
        tabs[mode] = [B.broadening(e) for e in range(len(evs))]
    for m in ("eager", "per_event"):
        for e in range(len(evs)):
            assert rel_err(tabs[m][e][:, 1:4], tabs["graph"][e][:, 1:4]) < 1e-13, (m, e)
    with pytest.raises(G.GlasmaError):
        B.run("persistent")
    for e, (gp, pp) in enumerate(zip(evs, pps)):
        n = gp.n
        a_fm = gp.L_fm / n
        a = a_fm / HBARC
        st, _, _ = O.glasma_init(n, gp.n_sheets, gp.g2mu_GeV * a, gp.m_ir_GeV * a, gp.seed, 0.125, tol=1e-14)
        P = O.particles_init(pp.n_particles, n, pp.mass_GeV * a, 0, 0.0, pp.p_max_GeV * a, pp.seed)
        n_form = max(1, int(round(pp.tau_form_fm / (0.125 * a_fm))))
        n_steps = int(np.ceil(gp.tau_end_fm / (0.125 * a_fm) - 1e-9))
        while st.step < n_form:
            st = O.field_step(st, 0.125)
        rows = []
        while st.step < n_steps:
            nx = O.field_step(st, 0.125)
            acc = O.push(P, st, nx, 0.125, pp.mass_GeV * a, 1, pp.integrator, pp.substeps, pp.interp)
            rows.append(acc[:3] / acc[3] / a ** 2)
            st = nx
        assert rel_err(tabs["graph"][e][1:, 1:4], np.array(rows)) < 1e-10, e
