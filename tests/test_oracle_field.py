"""Pins of the oracle's boost-invariant leapfrog (Sec. 1, "Glasma": lattice gauge
links and plaquettes in Milne coordinates)."""
import numpy as np
import pytest

import oracle as O


def rand_state(n, rng, scale=0.8, step=3, e_scale=0.5, phi_scale=0.4):
    st = O.State(n, step=step)
    for s in range(n * n):
        for d in range(2):
            st.U[s, d] = O.exp_i(scale * rng.standard_normal(8))
    st.E[...] = e_scale * rng.standard_normal((n * n, 2, 8))
    st.phi[...] = phi_scale * rng.standard_normal((n * n, 8))
    st.pi[...] = e_scale * rng.standard_normal((n * n, 8))
    return st


def gauss_free_state(n, rng, scale=0.8, step=3):
    """Random links and phi, E = 0, pi proportional to phi: G(x) = 0 exactly."""
    st = rand_state(n, rng, scale=scale, step=step)
    st.E[...] = 0
    st.pi[...] = 0.7 * st.phi
    return st


@pytest.mark.parametrize("expanding,tau", [(0, 1.0), (1, 0.6)])
def test_force_is_minus_group_gradient_of_potential(expanding, tau):
    """4x4 brute force: every link/site force equals a central finite difference of V."""
    rng = np.random.default_rng(10 + expanding)
    n = 4
    st = rand_state(n, rng)
    fE, fpi = O.force(n, tau, expanding, st.U, st.phi)
    h = 1e-6
    err = 0.0
    for s in range(n * n):
        for d in range(2):
            for a in range(8):
                e = np.zeros(8)
                e[a] = h
                Up, Um = st.U.copy(), st.U.copy()
                Up[s, d] = O.exp_i(e) @ st.U[s, d]
                Um[s, d] = O.exp_i(-e) @ st.U[s, d]
                g = (O.potential(n, tau, expanding, Up, st.phi) -
                     O.potential(n, tau, expanding, Um, st.phi)) / (2 * h)
                err = max(err, abs(-g - fE[s, d, a]))
        for a in range(8):
            pp, pm = st.phi.copy(), st.phi.copy()
            pp[s, a] += h
            pm[s, a] -= h
            g = (O.potential(n, tau, expanding, st.U, pp) -
                 O.potential(n, tau, expanding, st.U, pm)) / (2 * h)
            err = max(err, abs(-g - fpi[s, a]))
    assert err < 1e-7


def gauge_transform(st, Om):
    n = st.n
    out = st.copy()
    for s in range(n * n):
        x, y = s % n, s // n
        for d, sp in ((0, (x + 1) % n + n * y), (1, x + n * ((y + 1) % n))):
            out.U[s, d] = Om[s] @ st.U[s, d] @ Om[sp].conj().T
            out.E[s, d] = O.conj_by(Om[s], st.E[s, d])
        out.phi[s] = O.conj_by(Om[s], st.phi[s])
        out.pi[s] = O.conj_by(Om[s], st.pi[s])
    return out


@pytest.mark.parametrize("expanding", [0, 1])
def test_step_is_gauge_covariant(expanding):
    rng = np.random.default_rng(20)
    n, dtau = 6, 0.1
    st = rand_state(n, rng)
    Om = [O.exp_i(2.0 * rng.standard_normal(8)) for _ in range(n * n)]
    a = gauge_transform(O.field_step(st, dtau, expanding), Om)
    b = O.field_step(gauge_transform(st, Om), dtau, expanding)
    assert np.abs(a.U - b.U).max() < 1e-13
    assert np.abs(a.E - b.E).max() < 1e-12
    assert np.abs(a.phi - b.phi).max() < 1e-13
    assert np.abs(a.pi - b.pi).max() < 1e-12


@pytest.mark.parametrize("expanding", [0, 1])
def test_gauss_law_preserved(expanding):
    rng = np.random.default_rng(30)
    n, dtau = 8, 0.125
    st = gauss_free_state(n, rng)
    assert O.gauss_rel(st) < 1e-15
    for _ in range(60):
        st = O.field_step(st, dtau, expanding)
    assert np.abs(O.gauss(st)).max() < 1e-12
    assert O.gauss_rel(st) < 1e-13
    assert O.unitarity_all(st) < 1e-13


def hamiltonian_static(st_prev, st, st_next):
    """H at integer step n with E, pi averaged from n-1/2 and n+1/2 (static box)."""
    n = st.n
    E = 0.5 * (st.E + st_next.E)
    pi = 0.5 * (st.pi + st_next.pi)
    return O.energy(n, 1.0, 0, st.U, E, st.phi, pi).sum() * n * n


def test_energy_conserved_static_box_second_order():
    rng = np.random.default_rng(40)
    n = 6
    st0 = gauss_free_state(n, rng, scale=0.6)
    st0.E[...] = 0.3 * rng.standard_normal((n * n, 2, 8))
    devs = []
    for dtau in (0.04, 0.02):
        st = st0.copy()
        nxt = O.field_step(st, dtau, 0)
        H = []
        for _ in range(int(round(2.0 / dtau))):
            nn = O.field_step(nxt, dtau, 0)
            H.append(hamiltonian_static(st, nxt, nn))
            st, nxt = nxt, nn
        H = np.array(H)
        devs.append(np.abs(H - H[0]).max() / H[0])
    # bounded O(dtau^2) oscillation: halving dtau cuts the deviation ~4x
    assert devs[0] < 5e-3
    assert 3.0 < devs[0] / devs[1] < 5.0


def test_bjorken_balance_expanding():
    """d(tau eps)/dtau = -P_L with P_L = eps_T - eps_L, residual O(dtau^2)."""
    rng = np.random.default_rng(50)
    n = 6
    res = []
    for dtau in (0.02, 0.01):
        st = gauss_free_state(n, rng, scale=0.5, step=int(round(1.0 / dtau)))
        rng = np.random.default_rng(50)
        states = [st]
        for _ in range(int(round(0.4 / dtau)) + 2):
            states.append(O.field_step(states[-1], dtau, 1))
        te, PL = [], []
        for k in range(1, len(states) - 1):
            s, s1 = states[k], states[k + 1]
            tau = s.step * dtau
            e = O.energy(n, tau, 1, s.U, 0.5 * (s.E + s1.E), s.phi, 0.5 * (s.pi + s1.pi))
            te.append(tau * e.sum())
            PL.append((e[0] + e[1]) - (e[2] + e[3]))
        te, PL = np.array(te), np.array(PL)
        d = (te[2:] - te[:-2]) / (2 * dtau)
        res.append(np.abs(d + PL[1:-1]).max() / np.abs(PL).max())
    assert res[0] < 2e-2
    assert 3.5 < res[0] / res[1] < 4.8


@pytest.mark.parametrize("sector", ["E", "phi"])
def test_abelian_plane_wave_leapfrog_dispersion(sector):
    """Cartan-only small-amplitude wave: theta_n = A cos(k y) cos(omega n dtau) with the
    leapfrog dispersion sin(omega dtau / 2) = dtau sin(k / 2) (static box)."""
    n, dtau, A, m = 16, 0.1, 1e-4, 120
    k = 2 * np.pi * 3 / n
    w = 2.0 / dtau * np.arcsin(dtau * np.sin(k / 2))
    st = O.State(n, step=0)
    prof = np.array([np.cos(k * (s // n)) for s in range(n * n)])
    for s in range(n * n):
        st.U[s, 0] = st.U[s, 1] = np.eye(3)
    if sector == "E":
        th = np.zeros(8)
        for s in range(n * n):
            th[2] = A * prof[s]
            st.U[s, 0] = O.exp_i(th)
        st.E[:, 0, 2] = A * prof * (1 - np.cos(w * dtau)) / dtau
    else:
        st.phi[:, 2] = A * prof
        st.pi[:, 2] = A * prof * (1 - np.cos(w * dtau)) / dtau
    for _ in range(m):
        st = O.field_step(st, dtau, 0)
    if sector == "E":
        got = np.array([np.angle(st.U[s, 0][0, 0]) * 2 for s in range(n * n)])
    else:
        got = st.phi[:, 2]
    want = A * prof * np.cos(w * m * dtau)
    assert np.abs(got - want).max() < 1e-5 * A
