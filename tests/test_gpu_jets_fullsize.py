"""The jets workload at full size, in the launch configuration bench.py times: one 1024^2
event (L = 10 fm) with 1M massless partons along x in three ensembles (|p_x| = 2, 5, 10
GeV; 333,334 / 333,333 / 333,333), one parton per cell on average, sorted by cell every 16
steps and pushed in one shared launch per step.

The fields start from a seeded random state (links exp(i 0.7 x.t), E, phi, pi Gaussian)
instead of the MV initial condition, whose 1024^2 solve takes the oracle minutes; the
partons are formed at the first step.  The oracle evolves the fields itself for 40 steps
(two sorts on the GPU side) and pushes 200 sampled partons of each ensemble one by one.

- FP64 on the GPU: the sampled partons agree with the oracle to 1e-10 (positions modulo
  the lattice, momenta, rapidity, colour charge), the tables' counts are exact.
- FP32 on the GPU (the benchmark's precision, FP32 fields renormalised every step): the
  whole ensembles' <dp_i^2>(tau) within 1e-4 of their largest values against the FP64
  run (ensemble averages over 333k partons: a rounding-level shift of one parton's cell
  crossing moves them by ~1e-6)."""
import numpy as np
import pytest

import oracle as O
from gpu_common import rel_err

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_2307_07999_gb300")

N, L, STEP0, K = 1024, 10.0, 3, 40
HBARC = 0.1973269804
ENSEMBLES = [(2.0, 333334, 0x11AA01), (5.0, 333333, 0x11AA02), (10.0, 333333, 0x11AA03)]
N_SAMPLE = 200


def random_links(rng, count, scale):
    """exp(i scale x.t) for Gaussian x, by batched Hermitian eigendecomposition."""
    T = np.stack([O.generator(a) for a in range(8)])
    H = np.einsum("na,aij->nij", scale * rng.standard_normal((count, 8)), T)
    w, V = np.linalg.eigh(H)
    return np.einsum("nij,nj,nkj->nik", V, np.exp(1j * w), V.conj())


@pytest.fixture(scope="module")
def start():
    rng = np.random.default_rng(1024)
    st = O.State(N, step=STEP0)
    st.U[...] = random_links(rng, N * N * 2, 0.7).reshape(N * N, 2, 3, 3)
    st.E[...] = 0.4 * rng.standard_normal((N * N, 2, 8))
    st.phi[...] = 0.3 * rng.standard_normal((N * N, 8))
    st.pi[...] = 0.4 * rng.standard_normal((N * N, 8))
    return st


@pytest.fixture(scope="module")
def oracle_samples(start):
    a = (L / N) / HBARC
    rng = np.random.default_rng(7)
    samples = []
    for p, cnt, seed in ENSEMBLES:
        P = O.particles_init(cnt, N, 0.0, 1, p * a, p * a, seed)
        idx = np.sort(rng.choice(cnt, N_SAMPLE, replace=False))
        sub = O.Particles(N_SAMPLE)
        for k in ("x", "y", "eta", "px", "py", "peta", "Q", "p0"):
            getattr(sub, k)[...] = getattr(P, k)[idx]
        samples.append((idx, sub))
    st = start.copy()
    for _ in range(K):
        nx = O.field_step(st, 0.125)
        for _, sub in samples:
            O.push(sub, st, nx, 0.125, 0.0)
        st = nx
    return samples


def gpu_run(start, prec):
    g = G.Glasma(N, L, precision=prec, tau_end_fm=1.0, seed=1, reunit_every=(64 if prec else 0))
    g.set_state(start.U, start.E, start.phi, start.pi, STEP0)
    cs = []
    for p, cnt, seed in ENSEMBLES:
        c = G.CPIC(g, cnt, 0.0, 0.0, p_min_GeV=p, p_max_GeV=p, init_kind=1, bin_every=16, seed=seed)
        c.init()
        cs.append(c)
    G.push_many(cs, K)
    return g, cs


def test_jets_fullsize_fp64_sampled_against_oracle(start, oracle_samples):
    g, cs = gpu_run(start, 0)
    for (p, cnt, _), c, (idx, sub) in zip(ENSEMBLES, cs, oracle_samples):
        got = c.get_particles()
        for k in ("px", "py", "peta", "eta"):
            assert rel_err(got[k][idx], getattr(sub, k)) < 1e-10, (p, k)
        dx = np.abs(got["x"][idx] - sub.x)
        dy = np.abs(got["y"][idx] - sub.y)
        assert np.minimum(dx, N - dx).max() < 1e-10 and np.minimum(dy, N - dy).max() < 1e-10, p
        assert rel_err(got["Q"][idx], sub.Q) < 1e-10, p
        tab = c.broadening()
        assert tab.shape[0] == K + 1 and np.all(tab[1:, 4] == cnt)


def test_jets_fullsize_fp32_against_fp64(start):
    _, c64 = gpu_run(start, 0)
    _, c32 = gpu_run(start, 1)
    for (p, _, _), a, b in zip(ENSEMBLES, c32, c64):
        t32, t64 = a.broadening(), b.broadening()
        e = rel_err(t32[:, 1:4], t64[:, 1:4])
        print(f"p_x = {p} GeV: FP32 vs FP64 <dp^2> {e:.2e}")
        assert e < 1e-4, p
