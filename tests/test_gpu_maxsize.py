"""Large lattices, past 2^31 field elements (the plane offsets and the Fourier transforms
of the initial condition need 64-bit sizes), through the C ABI.

- 8192^2 in FP32 (64 planes x 67M sites = 4.3e9 reals per buffer): MV initial condition
  (FP64 Newton solve, 64-bit cuFFT plans), 12 field steps, monitors: every link solved,
  Gauss law and unitarity at FP32 rounding, finite energies.
- Translation invariance at 6200^2 (2.46e9 reals per buffer, 2.15e9 of them state): a state that repeats a
  10 x 10 random state 620 times in each direction evolves into the repetition of the
  oracle's evolution of the 10 x 10 state (FP32 2e-5 on sites sampled across the whole
  lattice, ragged tile edges and the periodic seams included).  The repeated state is
  written into a checkpoint blob of the large context (its body is the field buffer in
  the library's documented layout: 8 groups of 8 planes, interleaved per site, the last
  holding the plaquettes the next step rewrites); the result
  is read back in the canonical layout and compared with the oracle's small state.
"""
import ctypes as C

import numpy as np
import pytest

import oracle as O
from gpu_common import random_state, rel_err

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_2307_07999_gb300")


def host_gb_available():
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) / 2 ** 20
    except OSError:
        pass
    return 0.0


def test_8192_fp32_initial_condition_and_steps():
    n = 8192
    g = G.Glasma(n, 80.0, precision=G.GLASMA_FP32, tau_end_fm=1.0, seed=81, reunit_every=16)
    fails, mean_it, max_it = g.init()
    assert fails == 0 and 1.0 <= mean_it < 4.0
    g.step(12)
    d = g.diagnostics()
    assert d[7] == 0 and d[0] < 1e-5 and d[5] < 1e-5, d
    assert np.all(d[1:5] > 0) and np.all(np.isfinite(d[1:5]))


def field_body(blob, n, nbytes):
    """The field buffer (8 groups, n, n, 8 FP32 reals) of a checkpoint blob."""
    hdr = blob.size - nbytes
    return hdr, blob[hdr:hdr + 64 * n * n * 4].view(np.float32).reshape(8, n, n, 8)


def test_6200_translation_invariance_fp32():
    if host_gb_available() < 48:
        pytest.skip("needs ~20 GB of host memory for the 6200^2 state")
    p, reps, steps = 10, 620, 6
    n = p * reps
    align = lambda b: (b + 255) // 256 * 256
    small = random_state(p, seed=71, step=1)
    gs = G.Glasma(p, 1.0, precision=G.GLASMA_FP32, tau_end_fm=100.0)
    gs.set_state(small.U, small.E, small.phi, small.pi, small.step)
    _, body_s = field_body(gs.export_state(), p, align(64 * p * p * 4))
    gb = G.Glasma(n, 10.0, precision=G.GLASMA_FP32, tau_end_fm=100.0, seed=5)
    gb.init()  # any state at step 1: its blob carries the large context's header
    blob = gb.export_state()
    _, body_b = field_body(blob, n, align(64 * n * n * 4))
    for g_ in range(7):  # the state's groups, one at a time (keeps the host copy small)
        body_b[g_] = np.tile(body_s[g_], (reps, reps, 1))
    gb.import_state(blob)
    del blob, body_b
    gb.step(steps)
    st = small
    for _ in range(steps):
        st = O.field_step(st, 0.125)
    # the large state in the canonical layout, one field at a time (NULL skips the others),
    # against the oracle's small state at the sampled sites
    rng = np.random.default_rng(3)
    edge = [0, 1, n - 1, n - 2, 16 * 387, 16 * 387 + 7, 8 * 774 + 7]
    ys = np.concatenate([rng.integers(0, n, 300), edge, edge[::-1]])
    xs = np.concatenate([rng.integers(0, n, 300), edge[::-1], edge])
    sb, ss = xs + n * ys, xs % p + p * (ys % p)
    shapes = {"U": ((n * n, 2, 3, 3), np.complex128), "E": ((n * n, 2, 8), np.float64),
              "phi": ((n * n, 8), np.float64), "pi": ((n * n, 8), np.float64)}
    step = C.c_int32()
    for k, (shape, dt) in shapes.items():
        arr = np.zeros(shape, dtype=dt)
        ptrs = [arr.ctypes.data_as(C.c_void_p) if k == q else None for q in shapes]
        assert G.lib().glasma_get_state(gb.handle, *ptrs, C.byref(step)) == 0
        got = arr[sb].copy()
        del arr
        want = getattr(st, k)[ss]
        assert rel_err(got, want) < 2e-5, (k, rel_err(got, want))
    assert step.value == st.step
