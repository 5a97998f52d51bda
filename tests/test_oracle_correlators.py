"""Pins of the oracle's lattice-correlator estimators (Sec. 2, "Lattice correlators",
Eqs. 4 and 5): a closed form, the static (m -> infinity) and lightlike (p_x -> infinity)
limits of the independently written particle push for every site's charge, and gauge
invariance."""
import numpy as np
import pytest

import oracle as O


def rand_fields(n, rng, step=4):
    st = O.State(n, step=step)
    for s in range(n * n):
        for d in range(2):
            st.U[s, d] = O.exp_i(0.7 * rng.standard_normal(8))
    st.E[...] = 0.4 * rng.standard_normal((n * n, 2, 8))
    st.phi[...] = 0.4 * rng.standard_normal((n * n, 8))
    st.pi[...] = 0.4 * rng.standard_normal((n * n, 8))
    return st


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


def random_charges(np_, rng):
    Q0 = O.q0_cartan()
    return np.array([O.conj_by(O.haar(rng.standard_normal(18)), Q0) for _ in range(np_)])


def test_uniform_field_closed_form():
    """Static box, U = 1, a uniform E_x (any colour direction), phi = pi = 0: E stays
    uniform and every link stays exp(i t E), which commutes with E.  Both estimators
    then integrate E_x exactly: <dp_x^2> = (1/2) |e|^2 t^2, nothing along y or z."""
    rng = np.random.default_rng(0)
    n, dtau, m = 5, 0.1, 17
    e = rng.standard_normal(8)
    st = O.State(n, step=1)
    st.U[...] = np.eye(3)
    st.E[:, 0] = e
    C = O.Correlators(n, ox0=0.3)
    for _ in range(m):
        nx = O.field_step(st, dtau, 0)
        out = C.step(st, nx, dtau, 0)
        st = nx
    want = 0.5 * (e @ e) * (m * dtau) ** 2
    assert abs(out[0] - want) < 1e-12 * want and abs(out[3] - want) < 1e-12 * want
    assert np.abs(out[[1, 2, 4, 5]]).max() < 1e-24


@pytest.mark.parametrize("expanding", [0, 1])
def test_static_estimator_is_the_infinite_mass_push(expanding):
    """One heavy quark (m = 1e9 in lattice units, at rest) at the centre of every site,
    each with its own charge Q: its transverse momentum is Q.I_i of its site (the
    magnetic and Christoffel terms vanish with the velocity; p_z also in the static box),
    and the estimator is (1/2) sum_a I^a I^a averaged over sites."""
    rng = np.random.default_rng(1)
    n, dtau, m = 5, 0.1, 12
    st = rand_fields(n, rng, step=3)
    P = O.Particles(n * n)
    P.x[:] = np.arange(n * n) % n + 0.5
    P.y[:] = np.arange(n * n) // n + 0.5
    P.Q[...] = random_charges(n * n, rng)
    P.set_p0(1e9)
    C = O.Correlators(n)
    for _ in range(m):
        nx = O.field_step(st, dtau, expanding)
        out = C.step(st, nx, dtau, expanding)
        O.push(P, st, nx, dtau, 1e9, expanding)
        st = nx
    I = C.Istat
    for i, k in enumerate(("px", "py", "peta")):
        if k == "peta" and expanding:
            continue  # the Christoffel term acts on p_eta^ at any mass
        want = np.einsum("sa,sa->s", P.Q, I[:, i])
        got = getattr(P, k)
        assert np.abs(got - want).max() < 1e-7 * np.abs(want).max(), k
        assert abs(out[i] - 0.5 * (I[:, i] ** 2).sum() / (n * n)) < 1e-14 * out[i]


@pytest.mark.parametrize("expanding", [0, 1])
def test_lightlike_estimator_is_the_infinite_momentum_push(expanding):
    """A massless parton with p_x = 1e9 from offset 0.3 of every site (non-dyadic, so no
    crossing sits on a cell face), each with its charge Q0: its p_y is Q0.J_y of its start
    site, with J built from W F W^dag along the path; p_z too in the static box."""
    rng = np.random.default_rng(2)
    n, dtau, m = 5, 0.125, 30  # 50 steps of 1/8: six cell faces, once around the lattice
    st = rand_fields(n, rng, step=3)
    P = O.Particles(n * n)
    P.x[:] = np.arange(n * n) % n + 0.3
    P.y[:] = np.arange(n * n) // n + 0.5
    P.px[:] = 1e9
    Q0 = random_charges(n * n, rng)
    P.Q[...] = Q0
    P.set_p0(0.0)
    C = O.Correlators(n, ox0=0.3)
    for _ in range(m + 20):
        nx = O.field_step(st, dtau, expanding)
        out = C.step(st, nx, dtau, expanding)
        O.push(P, st, nx, dtau, 0.0, expanding)
        st = nx
    assert C.crossings(C.m, dtau) > n  # the paths went once around the periodic lattice
    J = C.J
    for i, k in ((1, "py"), (2, "peta")):
        if k == "peta" and expanding:
            continue
        want = np.einsum("sa,sa->s", Q0, J[:, i])
        assert np.abs(getattr(P, k) - want).max() < 1e-6 * np.abs(want).max(), k
        assert abs(out[3 + i] - 0.5 * (J[:, i] ** 2).sum() / (n * n)) < 1e-14 * out[3 + i]


@pytest.mark.parametrize("expanding", [0, 1])
def test_estimators_are_gauge_invariant(expanding):
    rng = np.random.default_rng(3)
    n, dtau, m = 5, 0.125, 14
    st = rand_fields(n, rng, step=3)
    Om = [O.exp_i(2 * rng.standard_normal(8)) for _ in range(n * n)]
    stg = gauge_transform(st, Om)
    A, B = O.Correlators(n, ox0=0.3), O.Correlators(n, ox0=0.3)
    for _ in range(m):
        nx, nxg = O.field_step(st, dtau, expanding), O.field_step(stg, dtau, expanding)
        a, b = A.step(st, nx, dtau, expanding), B.step(stg, nxg, dtau, expanding)
        st, stg = nx, nxg
        assert np.abs(a - b).max() < 1e-12 * np.abs(a).max()
