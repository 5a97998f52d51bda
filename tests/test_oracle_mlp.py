"""Pins of the oracle's warm-start network (the learned start of the tau = 0+ Newton
solve; the paper itself has no learned part)."""
import numpy as np

import oracle as O


def rand_weights(rng, scale=0.3):
    return {k: scale * rng.standard_normal(s) for k, s in O.MLP_SHAPES.items()}


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    w = rand_weights(rng)
    x = rng.standard_normal((5, 36))
    t = rng.standard_normal((5, 16))
    loss, g = O.mlp_loss_grad(x, t, w)
    h = 1e-6
    for k in w:
        flat = w[k].reshape(-1)
        for idx in rng.choice(flat.size, min(12, flat.size), replace=False):
            wp = {kk: v.copy() for kk, v in w.items()}
            wm = {kk: v.copy() for kk, v in w.items()}
            wp[k].reshape(-1)[idx] += h
            wm[k].reshape(-1)[idx] -= h
            fd = (O.mlp_loss_grad(x, t, wp)[0] - O.mlp_loss_grad(x, t, wm)[0]) / (2 * h)
            assert abs(fd - g[k].reshape(-1)[idx]) < 1e-8, (k, idx)
    # the loss is the mean squared error over batch and outputs
    y, _, _ = O.mlp_forward(x, w)
    assert abs(loss - ((y - t) ** 2).mean()) < 1e-14


def test_forward_special_cases():
    rng = np.random.default_rng(1)
    w = {k: np.zeros(s) for k, s in O.MLP_SHAPES.items()}
    w["b3"] = rng.standard_normal(16)
    y, h1, h2 = O.mlp_forward(rng.standard_normal((3, 36)), w)
    assert np.all(y == w["b3"]) and np.all(h1 == 0) and np.all(h2 == 0)


def test_target_vanishes_at_the_abelian_start_and_matches_the_solution():
    rng = np.random.default_rng(2)
    a, b = np.zeros(8), np.zeros(8)
    a[[2, 7]] = rng.standard_normal(2)
    b[[2, 7]] = rng.standard_normal(2)
    U1, U2 = O.exp_i(a), O.exp_i(b)
    U, it, res = O.ic_solve_link(U1, U2)
    # commuting links: U = U1 U2, so the offset, its series and the target all vanish
    assert np.abs(O.ic_delta(U1, U2, U)).max() < 1e-14
    assert np.abs(O.ic_series(U1, U2)).max() < 1e-14
    assert np.abs(O.ic_target(U1, U2, U)).max() < 1e-14
    # non-commuting: the start exp(i delta) U1 U2 reproduces the solution to O(delta^3)
    U1, U2 = O.exp_i(0.05 * rng.standard_normal(8)), O.exp_i(0.05 * rng.standard_normal(8))
    U, it, res = O.ic_solve_link(U1, U2)
    d = O.ic_delta(U1, U2, U)
    assert 1e-5 < np.abs(d).max() < 1e-2
    assert np.abs(O.exp_i(d) @ U1 @ U2 - U).max() < 10 * np.abs(d).max() ** 3
    assert np.allclose(O.ic_target(U1, U2, U), d - O.ic_series(U1, U2), atol=1e-15)


def test_series_start_is_exact_through_third_order():
    """delta - delta_s = O(a^4): halving the link fields divides the residual by ~16,
    while delta itself (second order) only falls by ~4.  A dropped or mis-signed
    term of the series would leave a second- or third-order residual (ratio 4 or 8)."""
    rng = np.random.default_rng(3)
    for _ in range(5):
        x1, x2 = rng.standard_normal(8), rng.standard_normal(8)
        r, dn = [], []
        for eps in (0.08, 0.04, 0.02):
            U1, U2 = O.exp_i(eps * x1), O.exp_i(eps * x2)
            U, it, res = O.ic_solve_link(U1, U2, tol=1e-15)
            r.append(np.linalg.norm(O.ic_delta(U1, U2, U) - O.ic_series(U1, U2)))
            dn.append(np.linalg.norm(O.ic_delta(U1, U2, U)))
        assert 3.0 < dn[0] / dn[1] < 5.0
        assert r[0] / r[1] > 12.0 and r[1] / r[2] > 13.0, r


def test_features_follow_the_lie_bracket():
    """Features of U1 = exp(i s t^1), U2 = exp(i s t^2): a1 = 2 sin(s/2) e_1,
    a2 = 2 sin(s/2) e_2, and c = i[a1 t^1, a2 t^2] = -a1 a2 t^3 from [t^1, t^2] = i t^3."""
    s = 0.3
    e1, e2 = np.zeros(8), np.zeros(8)
    e1[0], e2[1] = s, s
    U1, U2 = O.exp_i(e1), O.exp_i(e2)
    f = O.ic_features(U1, U2)
    a1, a2 = O.im_tl(U1), O.im_tl(U2)
    # exp(i s t^1) has 2 Im Tr[t^1 U] = 2 sin(s/2) and no other component
    assert np.allclose(a1, 2 * np.sin(s / 2) * np.eye(8)[0], atol=1e-15)
    assert np.allclose(f[:8], a1) and np.allclose(f[8:16], a2)
    c = f[16:24]
    assert np.allclose(c, -a1[0] * a2[1] * np.eye(8)[2], atol=1e-15)
    # cubic part from [t^1, t^3] = -i t^2 and [t^2, t^3] = i t^1
    c3 = c[2]
    cub1 = a1[0] * c3 * np.eye(8)[1]     # i[t^1, t^3] = t^2
    cub2 = -a2[1] * c3 * np.eye(8)[0]    # i[t^2, t^3] = -t^1
    assert np.allclose(f[24:32], -0.375 * cub1 - 0.125 * cub2, atol=1e-15)
    assert np.allclose(f[32:], [a1 @ a1, a2 @ a2, a1 @ a2, c @ c])
    assert np.allclose(O.ic_series(U1, U2), -0.5 * c + f[24:32])
