"""The learned warm start of the tau = 0+ link solve, through the C ABI: BF16/FP32
kernels against the FP64 oracle network, training on Newton-solved links, and the
iteration count of the warm-started solve on a fresh event."""
import numpy as np
import pytest

import oracle as O
from gpu_common import lattice_units, rel_err

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_2307_07999_gb300")
torch = pytest.importorskip("torch")


def bf16(a):
    t = torch.tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float32)
    return t.numpy().astype(np.float64)


def test_gradients_match_oracle():
    """One batch: loss and every gradient tensor against the FP64 network evaluated at
    the BF16-rounded weights and inputs (BF16 activations between layers: ~1e-2)."""
    rng = np.random.default_rng(0)
    net = G.WarmStartNet(seed=3)
    w, _ = net.params()
    w = {k: v.copy() for k, v in w.items()}
    w["W3"] = 0.3 * rng.standard_normal(w["W3"].shape).astype(np.float32)
    w["b1"] = 0.1 * rng.standard_normal(128).astype(np.float32)
    net.set_params(w)
    net.set_scales(1.0, 1.0)
    N = 301  # four full CTAs of 64 rows and a ragged fifth
    X = rng.uniform(-1, 1, (N, 36)).astype(np.float32)
    T = rng.standard_normal((N, 8)).astype(np.float32)
    loss, g = net.loss_grad(torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda"))
    wo = {k: bf16(v) if k.startswith("W") else v.astype(np.float64) for k, v in w.items()}
    t16 = np.zeros((N, 16))
    t16[:, :8] = T
    lo, go = O.mlp_loss_grad(bf16(X), t16, wo)
    assert abs(loss - lo) < 2e-2 * lo
    for k in go:
        e = rel_err(g[k], go[k])
        assert e < 3e-2, (k, e)


def test_features_and_targets_match_oracle():
    """Features and residual targets of every link of a weak-coupling event (where the
    GPU and oracle roots coincide) against the oracle's, computed from its own Wilson
    lines and Newton solution; FP32 storage of FP64 values."""
    n, L, seed = 32, 3.0, 4242
    a_fm, a, g2mua, mira = lattice_units(n, L)
    st, iters, fails = O.glasma_init(n, 10, g2mua, mira, seed, 0.125)
    assert fails == 0
    V1 = O.wilson_line(n, 10, g2mua, mira, seed, 0)
    V2 = O.wilson_line(n, 10, g2mua, mira, seed, 1)
    U1, U2 = O.pure_gauge_links(n, V1), O.pure_gauge_links(n, V2)
    Xo = np.array([O.ic_features(U1[s, d], U2[s, d]) for s in range(n * n) for d in range(2)])
    To = np.array([O.ic_target(U1[s, d], U2[s, d], st.U[s, d]) for s in range(n * n) for d in range(2)])
    g = G.Glasma(n, L, precision=1, tau_end_fm=1.0, seed=seed, newton_tol=1e-12)
    assert g.init()[0] == 0
    X, T = G.ic_dataset(g)
    X, T = X.cpu().numpy().astype(np.float64), T.cpu().numpy().astype(np.float64)
    assert np.abs(X - Xo).max() < 1e-6 * np.abs(Xo).max()
    assert np.abs(T - To).max() < 1e-6 * np.abs(To).max() + 1e-9


def event(n, L, seed, tol=1e-12):
    g = G.Glasma(n, L, precision=1, tau_end_fm=1.0, seed=seed, newton_tol=tol)
    return g


def test_training_reduces_loss_and_warm_start_cuts_iterations():
    n, L = 192, 10.0
    Xs, Ts = [], []
    for s in (101, 102, 103):
        g = event(n, L, s)
        assert g.init()[0] == 0
        X, T = G.ic_dataset(g)
        Xs.append(X)
        Ts.append(T)
    X = torch.cat(Xs)
    T = torch.cat(Ts)
    perm = torch.randperm(X.shape[0], device="cuda", generator=torch.Generator(device="cuda").manual_seed(0))
    X, T = X[perm].contiguous(), T[perm].contiguous()
    net = G.WarmStartNet(seed=5)
    net.fit_scales(X, T)
    l0, _ = net.loss_grad(X[:8192], T[:8192])
    loss = net.train(X, T, epochs=12, batch=2048, lr=2e-3)
    print(f"warm-start net: loss {l0:.3e} -> {loss:.3e}")
    assert loss < 0.1 * l0
    # a fresh event: same links, fewer Newton iterations
    cold = event(n, L, 999)
    f_c, it_c, mx_c = cold.init()
    warm = event(n, L, 999)
    f_w, it_w, mx_w = G.init_warm(warm, net)
    # the series alone: a network whose output layer is zero
    w, _ = net.params()
    w = {k: v.copy() for k, v in w.items()}
    w["W3"][:] = 0
    w["b3"][:] = 0
    zero = G.WarmStartNet(seed=5)
    zero.set_params(w)
    series = event(n, L, 999)
    f_s, it_s, mx_s = G.init_warm(series, zero)
    print(f"Newton iterations per link: cold {it_c:.3f} (max {mx_c}), series {it_s:.3f} (max {mx_s}), "
          f"series + network {it_w:.3f} (max {mx_w})")
    assert f_c == f_w == f_s == 0
    assert it_s < it_c
    assert it_w < 0.85 * it_c
    assert it_w < it_s
    Uc = cold.get_state()[0]
    for other in (warm, series):
        # FP32 state of the same roots (solved to 1e-12 in FP64)
        assert np.abs(Uc - other.get_state()[0]).max() < 1e-6
