"""Pins of the oracle's MV initial conditions (Sec. 1, "Glasma", Eq. 1 and the
boost-invariant matching at tau = 0+ that the paper defers to its companion paper)."""
import numpy as np
import scipy.linalg as sl

import oracle as O


def rand_su3(rng, scale=1.0):
    return sl.expm(1j * O.alg_to_mat(scale * rng.standard_normal(8)))


def test_fft_matches_numpy():
    rng = np.random.default_rng(0)
    for n in (8, 12, 15, 16):
        a = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        # oracle index s = x + n*y  <->  numpy a[y, x]
        assert np.allclose(O.fft2(a, -1), np.fft.fft2(a), atol=1e-11)
        assert np.allclose(O.fft2(a, +1), np.fft.ifft2(a) * n * n, atol=1e-11)


def test_poisson_solves_lattice_operator():
    # (-lattice Laplacian + m^2) Lambda = rho - (zero mode), checked with the stencil
    rng = np.random.default_rng(1)
    for n, m2 in ((16, 0.04), (12, 0.0)):
        rho = rng.standard_normal((n * n, 8))
        lam = O.poisson(n, m2, rho)
        L = lam.reshape(n, n, 8)
        lap = (np.roll(L, 1, 0) + np.roll(L, -1, 0) + np.roll(L, 1, 1) + np.roll(L, -1, 1) - 4 * L)
        lhs = (-lap + m2 * L).reshape(n * n, 8)
        assert np.abs(lhs - (rho - rho.mean(0))).max() < 1e-11


def test_pure_gauge_links_have_trivial_plaquettes():
    n = 8
    V = O.wilson_line(n, 3, 0.9, 0.2, 5, 0)
    for v in V:
        assert O.unitarity_dev(v) < 1e-13
    UA = O.pure_gauge_links(n, V)
    st = O.State(n)
    st.U[...] = UA
    # pure gauge: every plaquette is the identity, so the magnetic potential vanishes
    assert abs(O.potential(n, 1.0, 0, st.U, st.phi)) < 1e-12


def test_ic_abelian_exact_root():
    # commuting (Cartan) nucleus links: U = U1 U2 solves the matching condition
    rng = np.random.default_rng(2)
    for _ in range(5):
        a, b = np.zeros(8), np.zeros(8)
        a[[2, 7]] = rng.standard_normal(2)
        b[[2, 7]] = rng.standard_normal(2)
        U1, U2 = O.exp_i(a), O.exp_i(b)
        assert np.abs(O.ic_residual(U1, U2, U1 @ U2)).max() < 1e-15
        U, it, res = O.ic_solve_link(U1, U2, U_start=np.eye(3))
        assert it >= 0 and res < 1e-12


def test_ic_jacobian_matches_finite_differences():
    rng = np.random.default_rng(3)
    U1, U2, U = rand_su3(rng), rand_su3(rng), rand_su3(rng)
    J = O.ic_jacobian(U1, U2, U)
    h = 1e-6
    for b in range(8):
        e = np.zeros(8)
        e[b] = h
        rp = O.ic_residual(U1, U2, O.exp_i(e) @ U)
        rm = O.ic_residual(U1, U2, O.exp_i(-e) @ U)
        assert np.abs((rp - rm) / (2 * h) - J[:, b]).max() < 1e-8


def test_ic_solution_satisfies_condition():
    rng = np.random.default_rng(4)
    n = 8
    U1 = np.array([rand_su3(rng, 0.4) for _ in range(2 * n * n)]).reshape(n * n, 2, 3, 3)
    U2 = np.array([rand_su3(rng, 0.4) for _ in range(2 * n * n)]).reshape(n * n, 2, 3, 3)
    U, it, res, fails = O.ic_solve(n, U1, U2)
    assert fails == 0
    for l in range(2 * n * n):
        u = U.reshape(-1, 3, 3)[l]
        r = O.ic_residual(U1.reshape(-1, 3, 3)[l], U2.reshape(-1, 3, 3)[l], u)
        assert np.linalg.norm(r) <= 1e-12
        assert O.unitarity_dev(u) < 1e-12
        # the defining condition, restated with matrices: Tr[t^a (M - M^dag)] = 0
        M = (U1.reshape(-1, 3, 3)[l] + U2.reshape(-1, 3, 3)[l]) @ (np.eye(3) + u.conj().T)
        for a in range(8):
            assert abs(np.trace(O.generator(a) @ (M - M.conj().T))) < 3e-12


def test_pi0_weak_field_limit():
    # U^(A) = exp(i eps A^(A)):  pi(0) -> -i sum_i [A1_i, A2_i] + O(eps^3), the commutator
    # averaged over the two links of direction i that touch the site
    rng = np.random.default_rng(5)
    n = 6
    a1 = rng.standard_normal((n * n, 2, 8))
    a2 = rng.standard_normal((n * n, 2, 8))
    errs = []
    for eps in (1e-2, 5e-3):
        U1 = np.array([[O.exp_i(eps * a1[s, d]) for d in range(2)] for s in range(n * n)])
        U2 = np.array([[O.exp_i(eps * a2[s, d]) for d in range(2)] for s in range(n * n)])
        U, it, res, fails = O.ic_solve(n, U1, U2)
        assert fails == 0
        pi = O.pi0(n, U, U1, U2)
        lead = np.zeros((n * n, 8))
        for s in range(n * n):
            x, y = s % n, s // n
            C = np.zeros((3, 3), dtype=complex)
            for d in range(2):
                sm = ((x - 1) % n + n * y) if d == 0 else (x + n * ((y - 1) % n))
                for t in (s, sm):  # the two links of direction d touching site s
                    A, B = O.alg_to_mat(a1[t, d]), O.alg_to_mat(a2[t, d])
                    C += -0.5j * (A @ B - B @ A)
            lead[s] = O.mat_to_alg(C) * eps * eps
        errs.append(np.abs(pi - lead).max() / (eps * eps))
    # relative error of the leading term shrinks like eps
    assert errs[0] < 0.2 and errs[1] < 0.55 * errs[0]


def test_glasma_init_state():
    n, dtau = 8, 0.125
    st, iters, fails = O.glasma_init(n, 4, 0.5, 0.1, 11, dtau)
    assert fails == 0 and st.step == 1
    assert np.all(st.E == 0)
    # phi(tau_1) = dtau * tau_1/2 * pi(tau_1/2), Gauss law holds exactly
    assert np.allclose(st.phi, dtau * 0.5 * dtau * st.pi, atol=1e-15)
    assert O.gauss_rel(st) < 1e-14
    assert O.unitarity_all(st) < 1e-12
