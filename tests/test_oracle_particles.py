"""Pins of the oracle's colored particle-in-cell push (Sec. 1, "Probes in Glasma",
Eq. 2; the static and lightlike limits of Sec. 2, Eqs. 4 and 5)."""
import numpy as np
import pytest

import oracle as O


def vac_state(n, step=1):
    st = O.State(n, step=step)
    st.U[...] = np.eye(3)
    return st


def run(P, st, dtau, mass, m, expanding=1, hook=None):
    for _ in range(m):
        nx = O.field_step(st, dtau, expanding)
        if hook:
            hook(P, st, nx)
        O.push(P, st, nx, dtau, mass, expanding)
        st = nx
    return st


def make_particles(np_, n, rng, pscale=0.5, mass=0.7, peta=False):
    P = O.Particles(np_)
    P.x[:] = rng.uniform(0, n, np_)
    P.y[:] = rng.uniform(0, n, np_)
    P.px[:] = pscale * rng.standard_normal(np_)
    P.py[:] = pscale * rng.standard_normal(np_)
    if peta:
        P.peta[:] = pscale * rng.standard_normal(np_)
    Q0 = O.q0_cartan()
    for j in range(np_):
        P.Q[j] = O.conj_by(O.haar(rng.standard_normal(18)), Q0)
    P.set_p0(mass)
    return P


def test_free_streaming_static_box():
    rng = np.random.default_rng(1)
    n, dtau, mass, m = 8, 0.1, 0.7, 40
    P = make_particles(200, n, rng, mass=mass)
    P0 = P.copy()
    run(P, vac_state(n, 0), dtau, mass, m, expanding=0)
    assert np.all(P.px == P0.px) and np.all(P.py == P0.py) and np.all(P.peta == 0)
    pt = np.sqrt(mass ** 2 + P0.px ** 2 + P0.py ** 2)
    dx = (P0.x + m * dtau * P0.px / pt) % n
    d = np.abs(P.x - dx)
    assert np.minimum(d, n - d).max() < 1e-12
    assert np.abs(P.Q - P0.Q).max() < 1e-13


def test_free_particle_lab_pz_conserved_milne_first_order():
    """Zero field in Milne coordinates: the lab p_z of a free particle is constant;
    the explicit scheme conserves it to O(dtau)."""
    errs = []
    for dtau in (0.02, 0.01):
        P = O.Particles(1)
        P.px[:] = 0.3
        P.peta[:] = 0.8
        mass = 1.0
        P.set_p0(mass)
        st = vac_state(4, step=int(round(0.5 / dtau)))
        run(P, st, dtau, mass, int(round(1.0 / dtau)), expanding=1)
        pz = O.pz_lab(mass, P.px[0], P.py[0], P.peta[0], P.eta[0])
        errs.append(abs(pz - 0.8))
    assert errs[0] < 0.05
    assert 1.7 < errs[0] / errs[1] < 2.3


def pure_gauge_state(n, Om, step=1):
    st = O.State(n, step=step)
    for s in range(n * n):
        x, y = s % n, s // n
        st.U[s, 0] = Om[s] @ Om[(x + 1) % n + n * y].conj().T
        st.U[s, 1] = Om[s] @ Om[x + n * ((y + 1) % n)].conj().T
    return st


def test_pure_gauge_color_transport():
    rng = np.random.default_rng(2)
    n, dtau, mass = 6, 0.125, 0.5
    Om = [O.exp_i(2 * rng.standard_normal(8)) for _ in range(n * n)]
    P = make_particles(100, n, rng, pscale=0.8, mass=mass)
    P0 = P.copy()
    c0 = (np.floor(P0.x) + n * np.floor(P0.y)).astype(int)
    run(P, pure_gauge_state(n, Om, 0), dtau, mass, 60, expanding=0)
    assert np.abs(P.px - P0.px).max() < 1e-13 and np.abs(P.py - P0.py).max() < 1e-13
    c = (np.floor(P.x) + n * np.floor(P.y)).astype(int)
    assert np.count_nonzero(c != c0) > 50
    for j in range(P.np):
        W = Om[c[j]] @ Om[c0[j]].conj().T
        assert np.abs(P.Q[j] - O.conj_by(W, P0.Q[j])).max() < 1e-12


def rand_fields(n, rng, step=4):
    st = O.State(n, step=step)
    for s in range(n * n):
        for d in range(2):
            st.U[s, d] = O.exp_i(0.7 * rng.standard_normal(8))
    st.E[...] = 0.4 * rng.standard_normal((n * n, 2, 8))
    st.phi[...] = 0.4 * rng.standard_normal((n * n, 8))
    st.pi[...] = 0.4 * rng.standard_normal((n * n, 8))
    return st


@pytest.mark.parametrize("expanding", [0, 1])
def test_gauge_invariance_of_momenta(expanding):
    rng = np.random.default_rng(3)
    n, dtau, mass, m = 6, 0.1, 0.6, 30
    st = rand_fields(n, rng)
    P = make_particles(80, n, rng, mass=mass, peta=True)
    Om = [O.exp_i(2 * rng.standard_normal(8)) for _ in range(n * n)]
    stg = st.copy()
    for s in range(n * n):
        x, y = s % n, s // n
        for d, sp in ((0, (x + 1) % n + n * y), (1, x + n * ((y + 1) % n))):
            stg.U[s, d] = Om[s] @ st.U[s, d] @ Om[sp].conj().T
            stg.E[s, d] = O.conj_by(Om[s], st.E[s, d])
        stg.phi[s] = O.conj_by(Om[s], st.phi[s])
        stg.pi[s] = O.conj_by(Om[s], st.pi[s])
    Pg = P.copy()
    for j in range(P.np):
        Pg.Q[j] = O.conj_by(Om[int(P.x[j]) + n * int(P.y[j])], P.Q[j])
    run(P, st, dtau, mass, m, expanding)
    run(Pg, stg, dtau, mass, m, expanding)
    for k in ("px", "py", "peta", "x", "y", "eta"):
        assert np.abs(getattr(P, k) - getattr(Pg, k)).max() < 1e-11
    for j in range(P.np):
        c = int(P.x[j]) + n * int(P.y[j])
        assert np.abs(Pg.Q[j] - O.conj_by(Om[c], P.Q[j])).max() < 1e-11


def test_casimirs_conserved():
    rng = np.random.default_rng(4)
    n, dtau, mass = 6, 0.1, 0.3
    st = rand_fields(n, rng)
    P = make_particles(60, n, rng, pscale=1.0, mass=mass, peta=True)
    run(P, st, dtau, mass, 80, expanding=1)
    for j in range(P.np):
        q2, q3 = O.casimirs(P.Q[j])
        assert abs(q2 - 4.0) < 1e-12 and abs(q3 - 10.0 / 3.0) < 1e-12


def test_constant_cartan_electric_field():
    """Uniform E_x = e t^3 (static box): p_x grows by Q^3 e per unit time, exactly; the
    position follows the relativistic closed form to first order in dtau."""
    e, mass, T = 0.3, 0.5, 4.0
    errs = []
    for dtau in (0.02, 0.01):
        st = vac_state(8, 0)
        st.E[:, 0, 2] = e
        rng = np.random.default_rng(5)
        P = make_particles(20, 8, rng, pscale=0.0, mass=mass)
        P0 = P.copy()
        m = int(round(T / dtau))
        run(P, st, dtau, mass, m, expanding=0)
        q3 = P0.Q[:, 2]
        assert np.abs(P.px - q3 * e * m * dtau).max() < 1e-12
        assert np.abs(P.Q[:, 2] - q3).max() < 1e-13
        F = q3 * e
        xc = P0.x + (np.sqrt(mass ** 2 + (F * T) ** 2) - mass) / F
        d = np.abs((P.x - xc) % 8)
        errs.append(np.minimum(d, 8 - d).max())
    assert errs[0] < 0.05 and 1.7 < errs[0] / errs[1] < 2.3


def uniform_bz_state(n, k=1):
    """U_x(x,y) = exp(-i b y t^3), U_y = 1 except the twist row, b = 4 pi k / n^2: every
    plaquette equals exp(i b t^3)."""
    b = 4 * np.pi * k / n ** 2
    st = vac_state(n, 0)
    for s in range(n * n):
        x, y = s % n, s // n
        th = np.zeros(8)
        th[2] = -b * y
        st.U[s, 0] = O.exp_i(th)
        if y == n - 1:
            th[2] = b * n * x
            st.U[s, 1] = O.exp_i(th)
    return st, b


def test_uniform_bz_is_uniform_and_cyclotron_first_order():
    n = 24
    st, b = uniform_bz_state(n)
    bz = -2 * np.sin(b / 2)  # B_z = -F_xy, F_xy = ImTL(exp(i b t^3)) = 2 sin(b/2) t^3
    for cx, cy in ((3, 5), (0, 0), (n - 1, n - 1), (10, n - 1)):
        F = O.gather(st, st, cx, cy, 1.0, expanding=0)
        assert abs(F[5][2] - bz) < 1e-14 and np.abs(np.delete(F[5], 2)).max() < 1e-14
        assert np.abs(F[:5]).max() < 1e-14
    mass, p0, T = 0.4, 0.3, 6.0
    Q0 = O.q0_cartan()
    errs = []
    for dtau in (0.01, 0.005):
        P = O.Particles(1)
        P.x[:] = 12.3
        P.y[:] = 11.7
        P.px[:] = p0
        P.Q[0] = Q0
        P.set_p0(mass, expanding=0)
        run(P, uniform_bz_state(n)[0], dtau, mass, int(round(T / dtau)), expanding=0)
        w = Q0[2] * bz / np.sqrt(mass ** 2 + p0 ** 2)  # dp/dt = Q.Bz (p_y, -p_x)/p^tau
        want = p0 * np.array([np.cos(w * T), -np.sin(w * T)])
        errs.append(np.hypot(P.px[0] - want[0], P.py[0] - want[1]) / p0)
    assert errs[0] < 0.05 and 1.7 < errs[0] / errs[1] < 2.3


def _static_run(dtau, t0=0.4, t1=2.4, seed=6):
    rng = np.random.default_rng(seed)
    n, mass = 6, 1e8
    st = rand_fields(n, rng, step=int(round(t0 / dtau)))
    P = make_particles(40, n, rng, pscale=0.0, mass=mass)
    Q = P.Q.copy()
    cells = [(int(P.x[j]), int(P.y[j])) for j in range(P.np)]
    integ = np.zeros((P.np, 3, 8))

    def hook(P_, old, new):
        tau = old.step * dtau
        for j, (cx, cy) in enumerate(cells):
            # E at the site: the two links touching c, time-centred, transported
            s = cx + n * cy
            for d, sm in ((0, (cx - 1) % n + n * cy), (1, cx + n * ((cy - 1) % n))):
                Ec = 0.5 * (old.E[s, d] + new.E[s, d])
                Em = 0.5 * (old.E[sm, d] + new.E[sm, d])
                Um = old.U[sm, d]
                Emt = O.mat_to_alg(Um.conj().T @ O.alg_to_mat(Em) @ Um)
                integ[j, d] += dtau * 0.5 * (Ec + Emt) / tau
            integ[j, 2] += dtau * 0.5 * (old.pi[s] + new.pi[s])

    run(P, st, dtau, mass, int(round((t1 - t0) / dtau)), expanding=1, hook=hook)
    want = np.einsum("ja,jia->ji", Q, integ)
    # longitudinal: the lab p_z; in Milne coordinates the eta drift cancels the
    # Christoffel term, so p_z (not p_eta^) integrates Q.E_z
    pz = np.array([O.pz_lab(mass, P.px[j], P.py[j], P.peta[j], P.eta[j]) for j in range(P.np)])
    return np.stack([P.px, P.py, pz], 1), want, Q, integ, rng


def test_static_limit_equals_electric_field_integral():
    """m -> infinity, p = 0: delta p_i = sum_n dtau Q.E_i(c0, tau_n) (Eq. 4 per particle):
    exact for the transverse components, first order in dtau for the lab p_z; the Q
    average of (Q.v)^2 is Tr(v^2) (Eq. 4 with <Q^a Q^b> = delta^ab / 2)."""
    got, want, Q, integ, rng = _static_run(0.1)
    assert np.abs(got[:, :2] - want[:, :2]).max() < 1e-6 * np.abs(want[:, :2]).max()
    e1 = np.abs(got[:, 2] - want[:, 2]).max()
    got2, want2, *_ = _static_run(0.05)
    e2 = np.abs(got2[:, 2] - want2[:, 2]).max()
    assert e1 < 0.1 * np.abs(want[:, 2]).max() and 1.6 < e1 / e2 < 2.4
    v = integ[0, 0]
    Q0 = O.q0_cartan()
    qs = np.array([O.conj_by(O.haar(rng.standard_normal(18)), Q0) for _ in range(20000)])
    proj = (qs @ v) ** 2
    assert abs(proj.mean() - 0.5 * v @ v) < 5 * proj.std() / np.sqrt(len(qs))


def test_lightlike_limit_force_combination():
    """v_x -> 1: the kicks on p_y and p_eta are Q.(E_y - B_z) and Q.(E_z + B_y) (Eq. 5)."""
    rng = np.random.default_rng(7)
    n, dtau, mass = 6, 0.1, 0.0
    st = rand_fields(n, rng)
    P = make_particles(30, n, rng, pscale=0.0, mass=mass)
    P.px[:] = 1e7
    P.set_p0(mass)
    nx = O.field_step(st, dtau, 1)
    Pb = P.copy()
    O.push(P, st, nx, dtau, mass, 1)
    tau = st.step * dtau
    for j in range(P.np):
        F = O.gather(st, nx, int(Pb.x[j]), int(Pb.y[j]), dtau, expanding=1)
        q = Pb.Q[j]
        assert abs((P.py[j] - Pb.py[j]) - dtau * q @ (F[1] - F[5])) < 1e-9
        assert abs((P.peta[j] - Pb.peta[j]) - dtau * q @ (F[2] + F[4])) < 1e-9
        assert abs((P.px[j] - Pb.px[j]) - dtau * q @ F[0]) < 1e-9 * 1e7


def test_particle_init_distributions():
    n = 32
    P = O.particles_init(20000, n, 0.5, 0, 0.0, 2.0, 1234)
    f, d = O.structure_constants()
    Q = P.Q
    N = len(Q)
    q2 = (Q ** 2).sum(1)
    q3 = np.einsum("abc,ja,jb,jc->j", d, Q, Q, Q)
    assert np.abs(q2 - 4).max() < 1e-12 and np.abs(q3 - 10 / 3).max() < 1e-12
    assert np.abs(Q.mean(0)).max() < 5 * np.sqrt(0.5 / N)
    assert np.abs(Q.T @ Q / N - 0.5 * np.eye(8)).max() < 5 * np.sqrt(1.0 / N)
    m3 = np.einsum("ja,jb,jc->abc", Q, Q, Q) / N
    assert np.abs(m3 - d / 4).max() < 6 * np.sqrt(2.0 / N)
    assert P.x.min() >= 0 and P.x.max() < n and abs(P.x.mean() - n / 2) < 5 * n / np.sqrt(12 * N)
    pt = np.hypot(P.px, P.py)
    assert pt.max() <= 2.0 and abs(pt.mean() - 1.0) < 5 * 2 / np.sqrt(12 * N)
    assert np.all(P.eta == 0) and np.all(P.peta == 0)


# ---------------------------------------------------------------- Boris integrator
def run_int(P, st, dtau, mass, m, expanding, integrator):
    for _ in range(m):
        nx = O.field_step(st, dtau, expanding)
        O.push(P, st, nx, dtau, mass, expanding, integrator)
        st = nx
    return st


def test_boris_uniform_bz_norm_exact_and_cyclotron_second_order():
    """Pure magnetic field: the Boris rotation keeps |p| to rounding at any step, and
    the orbit converges at second order (the explicit kick: first order, |p| grows)."""
    n = 24
    bz = -2 * np.sin(uniform_bz_state(n)[1] / 2)
    mass, p0, T = 0.4, 0.3, 6.0
    Q0 = O.q0_cartan()
    w = Q0[2] * bz / np.sqrt(mass ** 2 + p0 ** 2)
    errs = []
    for dtau in (0.04, 0.02):
        P = O.Particles(1)
        P.x[:], P.y[:], P.px[:] = 12.3, 11.7, p0
        P.Q[0] = Q0
        P.set_p0(mass, expanding=0)
        run_int(P, uniform_bz_state(n)[0], dtau, mass, int(round(T / dtau)), 0, 1)
        assert abs(np.hypot(P.px[0], P.py[0]) - p0) < 1e-14
        want = p0 * np.array([np.cos(w * T), -np.sin(w * T)])
        errs.append(np.hypot(P.px[0] - want[0], P.py[0] - want[1]) / p0)
    assert errs[0] < 0.01 and 3.5 < errs[0] / errs[1] < 4.5, errs
    P = O.Particles(1)
    P.x[:], P.y[:], P.px[:] = 12.3, 11.7, p0
    P.Q[0] = Q0
    P.set_p0(mass, expanding=0)
    run_int(P, uniform_bz_state(n)[0], 0.04, mass, 150, 0, 0)
    assert np.hypot(P.px[0], P.py[0]) > p0 * (1 + 1e-4)


def test_boris_equals_explicit_without_magnetic_field():
    """Uniform Cartan E_x, no B: both integrators give p_x = p_0 + Q^3 e t exactly and
    the same positions."""
    e, mass, dtau, m = 0.3, 0.5, 0.02, 120
    st = vac_state(8, 0)
    st.E[:, 0, 2] = e
    rng = np.random.default_rng(5)
    P = make_particles(20, 8, rng, pscale=0.2, mass=mass)
    Pb = P.copy()
    run_int(P, st, dtau, mass, m, 0, 0)
    run_int(Pb, st, dtau, mass, m, 0, 1)
    for k in ("px", "py", "peta", "x", "y"):
        assert np.abs(getattr(P, k) - getattr(Pb, k)).max() < 1e-12, k


def test_boris_milne_free_particle_peta_exact():
    """Zero field in Milne coordinates: p_eta^ = tau p^eta falls as 1/tau exactly (the
    covariant p_eta = tau^2 p^eta is conserved); the Boris step applies that decay
    exactly, the explicit kick to first order."""
    dtau, mass, tau0, T = 0.02, 1.0, 0.5, 1.0
    res = {}
    for integrator in (0, 1):
        P = O.Particles(1)
        P.px[:] = 0.3
        P.peta[:] = 0.8
        P.set_p0(mass)
        st = vac_state(4, step=int(round(tau0 / dtau)))
        run_int(P, st, dtau, mass, int(round(T / dtau)), 1, integrator)
        res[integrator] = P.peta[0]
    want = 0.8 * tau0 / (tau0 + T)
    assert abs(res[1] - want) < 1e-14
    assert abs(res[0] - want) > 1e-4


@pytest.mark.parametrize("expanding", [0, 1])
def test_boris_is_gauge_invariant(expanding):
    rng = np.random.default_rng(13)
    n, dtau, mass, m = 6, 0.1, 0.6, 30
    st = rand_fields(n, rng)
    P = make_particles(60, n, rng, mass=mass, peta=True)
    Om = [O.exp_i(2 * rng.standard_normal(8)) for _ in range(n * n)]
    stg = st.copy()
    for s in range(n * n):
        x, y = s % n, s // n
        for d, sp in ((0, (x + 1) % n + n * y), (1, x + n * ((y + 1) % n))):
            stg.U[s, d] = Om[s] @ st.U[s, d] @ Om[sp].conj().T
            stg.E[s, d] = O.conj_by(Om[s], st.E[s, d])
        stg.phi[s] = O.conj_by(Om[s], st.phi[s])
        stg.pi[s] = O.conj_by(Om[s], st.pi[s])
    Pg = P.copy()
    for j in range(P.np):
        Pg.Q[j] = O.conj_by(Om[int(P.x[j]) + n * int(P.y[j])], P.Q[j])
    run_int(P, st, dtau, mass, m, expanding, 1)
    run_int(Pg, stg, dtau, mass, m, expanding, 1)
    for k in ("px", "py", "peta", "x", "y", "eta"):
        assert np.abs(getattr(P, k) - getattr(Pg, k)).max() < 1e-11


# ---------------------------------------------------------------- sub-cycled particle steps
def run_sub(P, st, dtau, mass, m, expanding, integrator, substeps):
    for _ in range(m):
        nx = O.field_step(st, dtau, expanding)
        O.push(P, st, nx, dtau, mass, expanding, integrator, substeps)
        st = nx
    return st


@pytest.mark.parametrize("integrator", [0, 1])
def test_substeps_equal_finer_steps_in_static_fields(integrator):
    """In the static box with fields that do not evolve (a uniform Cartan B_z: every
    plaquette equal, no staple force, E = 0 so the links stay put), s sub-steps of dtau/s
    within one field step are the same particle steps as s field steps of dtau/s
    (cyclotron orbits crossing cells, colour carried by the links): identical to
    rounding, for either kick."""
    n, mass, dtau, s, m = 16, 0.5, 0.08, 4, 25
    st = uniform_bz_state(n, k=3)[0]
    rng = np.random.default_rng(21)
    P = make_particles(40, n, rng, pscale=0.3, mass=mass)
    P.set_p0(mass, expanding=0)
    Pf = P.copy()
    run_sub(P, st, dtau, mass, m, 0, integrator, s)
    run_sub(Pf, st, dtau / s, mass, m * s, 0, integrator, 1)
    for k in ("px", "py", "peta", "x", "y", "eta", "Q"):
        assert np.abs(getattr(P, k) - getattr(Pf, k)).max() < 1e-12, k


def test_substeps_cyclotron_error_falls_as_one_over_s():
    """Uniform B_z, explicit kick (first order): at a fixed field step the orbit error
    falls as 1/s with the sub-steps."""
    n = 24
    bz = -2 * np.sin(uniform_bz_state(n)[1] / 2)
    mass, p0, T, dtau = 0.4, 0.3, 6.0, 0.04
    Q0 = O.q0_cartan()
    w = Q0[2] * bz / np.sqrt(mass ** 2 + p0 ** 2)
    want = p0 * np.array([np.cos(w * T), -np.sin(w * T)])
    errs = []
    for s in (1, 4):
        P = O.Particles(1)
        P.x[:], P.y[:], P.px[:] = 12.3, 11.7, p0
        P.Q[0] = Q0
        P.set_p0(mass, expanding=0)
        run_sub(P, uniform_bz_state(n)[0], dtau, mass, int(round(T / dtau)), 0, 0, s)
        errs.append(np.hypot(P.px[0] - want[0], P.py[0] - want[1]) / p0)
    assert 3.5 < errs[0] / errs[1] < 4.5, errs


@pytest.mark.parametrize("s", [1, 3, 8])
def test_substeps_milne_free_particle(s):
    """Zero field in Milne coordinates: with the Boris kick p_eta^ = p_eta^(tau0) tau0/tau
    exactly for any number of sub-steps (the half-step decays telescope only if every
    sub-step starts at its own tau_k); the explicit kick's error falls as 1/s; the
    transverse motion is a straight line at constant speed."""
    dtau, mass, tau0, T = 0.02, 1.0, 0.5, 1.0
    m = int(round(T / dtau))
    want = 0.8 * tau0 / (tau0 + T)
    errs = {}
    for integrator in (0, 1):
        P = O.Particles(1)
        P.x[:], P.px[:], P.peta[:] = 1.25, 0.3, 0.8
        P.set_p0(mass)
        run_sub(P, vac_state(4, step=int(round(tau0 / dtau))), dtau, mass, m, 1, integrator, s)
        errs[integrator] = abs(P.peta[0] - want)
        assert abs(P.px[0] - 0.3) < 1e-15 and P.py[0] == 0.0
    assert errs[1] < 1e-14
    P1 = O.Particles(1)
    P1.px[:], P1.peta[:] = 0.3, 0.8
    P1.set_p0(mass)
    run_sub(P1, vac_state(4, step=int(round(tau0 / dtau))), dtau, mass, m, 1, 0, 1)
    assert abs(errs[0] * s / abs(P1.peta[0] - want) - 1.0) < 0.05


def test_substeps_are_gauge_invariant():
    rng = np.random.default_rng(17)
    n, dtau, mass, m = 6, 0.1, 0.6, 20
    st = rand_fields(n, rng)
    P = make_particles(60, n, rng, mass=mass, peta=True)
    Om = [O.exp_i(2 * rng.standard_normal(8)) for _ in range(n * n)]
    stg = st.copy()
    for s in range(n * n):
        x, y = s % n, s // n
        for d, sp in ((0, (x + 1) % n + n * y), (1, x + n * ((y + 1) % n))):
            stg.U[s, d] = Om[s] @ st.U[s, d] @ Om[sp].conj().T
            stg.E[s, d] = O.conj_by(Om[s], st.E[s, d])
        stg.phi[s] = O.conj_by(Om[s], st.phi[s])
        stg.pi[s] = O.conj_by(Om[s], st.pi[s])
    Pg = P.copy()
    for j in range(P.np):
        Pg.Q[j] = O.conj_by(Om[int(P.x[j]) + n * int(P.y[j])], P.Q[j])
    run_sub(P, st, dtau, mass, m, 1, 1, 3)
    run_sub(Pg, stg, dtau, mass, m, 1, 1, 3)
    for k in ("px", "py", "peta", "x", "y", "eta"):
        assert np.abs(getattr(P, k) - getattr(Pg, k)).max() < 1e-11


# ---------------------------------------------------------------- cloud-in-cell gather
def test_cic_exact_for_affine_abelian_fields():
    """Links at unity, E_x, E_y, pi affine in (x, y) away from the periodic seam: the site
    average of the link fields is affine again (E_x(X, Y) = e0 + g_x (X - 1/2) + g_y Y, E_y
    with Y - 1/2), and bilinear weights reproduce an affine function exactly, so the
    cloud-in-cell field at the particle equals the closed form at its position; the
    nearest-grid-point field is the value at the cell's corner site."""
    n = 16
    rng = np.random.default_rng(31)
    st = vac_state(n, step=3)
    e0, gx, gy = rng.standard_normal((3, 3, 8))
    for s in range(n * n):
        X, Y = s % n, s // n
        st.E[s, 0] = e0[0] + gx[0] * X + gy[0] * Y
        st.E[s, 1] = e0[1] + gx[1] * X + gy[1] * Y
        st.pi[s] = e0[2] + gx[2] * X + gy[2] * Y
    for _ in range(20):
        x, y = rng.uniform(3, n - 4, 2)
        cx, cy = int(x), int(y)
        F = O.gather_cic(st, st, cx, cy, x - cx, y - cy, 0.1, expanding=0)
        assert np.abs(F[0] - (e0[0] + gx[0] * (x - 0.5) + gy[0] * y)).max() < 1e-12
        assert np.abs(F[1] - (e0[1] + gx[1] * x + gy[1] * (y - 0.5))).max() < 1e-12
        assert np.abs(F[2] - (e0[2] + gx[2] * x + gy[2] * y)).max() < 1e-12
        assert np.abs(F[3:]).max() < 1e-14
        G0 = O.gather(st, st, cx, cy, 0.1, expanding=0)
        assert np.abs(G0[0] - (e0[0] + gx[0] * (cx - 0.5) + gy[0] * cy)).max() < 1e-12


def test_cic_pure_gauge_of_uniform_fields_is_uniform():
    """A gauge transform of uniform fields (U_i(x) = W(x) W(x+i)^dag, every field
    W(x) F0 W(x)^dag): every site's fields carried to the cell's site are W(c) F0 W(c)^dag,
    so the cloud-in-cell gather equals the nearest-grid-point one at any offset.  This fixes
    the direction of every transport, the diagonal site's path included."""
    n = 8
    rng = np.random.default_rng(41)
    Wg = [O.exp_i(1.5 * rng.standard_normal(8)) for _ in range(n * n)]
    Ex, Ey, Pz, Ph = rng.standard_normal((4, 8))
    st = vac_state(n, step=3)
    for s in range(n * n):
        X, Y = s % n, s // n
        for d, sp in ((0, (X + 1) % n + n * Y), (1, X + n * ((Y + 1) % n))):
            st.U[s, d] = Wg[s] @ Wg[sp].conj().T
        st.E[s, 0] = O.conj_by(Wg[s], Ex)
        st.E[s, 1] = O.conj_by(Wg[s], Ey)
        st.pi[s] = O.conj_by(Wg[s], Pz)
        st.phi[s] = O.conj_by(Wg[s], Ph)
    for _ in range(10):
        cx, cy = rng.integers(0, n, 2)
        ox, oy = rng.uniform(0, 1, 2)
        F = O.gather_cic(st, st, cx, cy, ox, oy, 0.1, expanding=0)
        G0 = O.gather(st, st, cx, cy, 0.1, expanding=0)
        assert np.abs(F - G0).max() < 1e-12
        c = cx + n * cy
        assert np.abs(F[0] - O.conj_by(Wg[c], Ex)).max() < 1e-12


def test_cic_force_continuous_across_faces():
    """Random non-abelian fields: crossing an x face the contracted force is continuous
    (the charge is carried across by the same link that carries the fields), while the
    nearest-grid-point force jumps; crossing a y face the force jumps only by the
    plaquette holonomy of the diagonal site's two paths, a second-order amount that falls
    fourfold when the fields are halved."""
    n = 8
    rng = np.random.default_rng(51)

    def fields(scale):
        r = np.random.default_rng(52)
        st = O.State(n, step=3)
        for s in range(n * n):
            for d in range(2):
                st.U[s, d] = O.exp_i(scale * r.standard_normal(8))
        st.E[...] = scale * r.standard_normal((n * n, 2, 8))
        st.phi[...] = scale * r.standard_normal((n * n, 8))
        st.pi[...] = scale * r.standard_normal((n * n, 8))
        return st

    Q = O.conj_by(O.haar(rng.standard_normal(18)), O.q0_cartan())
    st = fields(0.3)
    cx, cy, oy, eps = 3, 4, 0.37, 1e-9
    before = O.gather_cic(st, st, cx, cy, 1 - eps, oy, 0.1, expanding=0) @ Q
    Qn = O.transport(st.U[cx + n * cy, 0], Q)
    after = O.gather_cic(st, st, cx + 1, cy, 0.0, oy, 0.1, expanding=0) @ Qn
    assert np.abs(before - after).max() < 1e-7
    ngp_jump = np.abs(O.gather(st, st, cx, cy, 0.1, 0) @ Q - O.gather(st, st, cx + 1, cy, 0.1, 0) @ Qn).max()
    assert ngp_jump > 1e-2
    jumps = []
    for scale in (0.2, 0.1):
        st = fields(scale)
        ox = 0.6
        b = O.gather_cic(st, st, cx, cy, ox, 1 - eps, 0.1, expanding=0) @ Q
        Qn = O.transport(st.U[cx + n * cy, 1], Q)
        a = O.gather_cic(st, st, cx, cy + 1, ox, 0.0, 0.1, expanding=0) @ Qn
        jumps.append(np.abs(b - a).max())
    assert 3.0 < jumps[0] / jumps[1] < 5.5, jumps


def test_cic_push_is_gauge_invariant():
    rng = np.random.default_rng(61)
    n, dtau, mass, m = 6, 0.1, 0.6, 20
    st = rand_fields(n, rng)
    P = make_particles(60, n, rng, mass=mass, peta=True)
    Om = [O.exp_i(2 * rng.standard_normal(8)) for _ in range(n * n)]
    stg = st.copy()
    for s in range(n * n):
        x, y = s % n, s // n
        for d, sp in ((0, (x + 1) % n + n * y), (1, x + n * ((y + 1) % n))):
            stg.U[s, d] = Om[s] @ st.U[s, d] @ Om[sp].conj().T
            stg.E[s, d] = O.conj_by(Om[s], st.E[s, d])
        stg.phi[s] = O.conj_by(Om[s], st.phi[s])
        stg.pi[s] = O.conj_by(Om[s], st.pi[s])
    Pg = P.copy()
    for j in range(P.np):
        Pg.Q[j] = O.conj_by(Om[int(P.x[j]) + n * int(P.y[j])], P.Q[j])
    for _ in range(m):
        nx, nxg = O.field_step(st, dtau, 1), O.field_step(stg, dtau, 1)
        O.push(P, st, nx, dtau, mass, 1, 1, 2, 1)
        O.push(Pg, stg, nxg, dtau, mass, 1, 1, 2, 1)
        st, stg = nx, nxg
    for k in ("px", "py", "peta", "x", "y", "eta"):
        assert np.abs(getattr(P, k) - getattr(Pg, k)).max() < 1e-11
