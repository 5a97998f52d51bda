"""glasma_diagnostics_noalloc: the field monitors for callers that cannot allocate
device memory (they own the field buffer; the library keeps its reduction scratch
in a static device array).  Checked through the C ABI against glasma_diagnostics
on the same state, on two calls in a row.  This file sorts last so that a run
stopping at its first failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest

from gpu_common import random_state, rel_err

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_2307_07999_gb300")
torch = pytest.importorskip("torch")


def plane_buffer(st, prec):
    """The canonical state in the library's plane layout (56 planes, grouped by eight and
    interleaved per site), on the device (caller-owned)."""
    n = st.n
    ns = n * n
    f = np.zeros((56, ns))
    for d in range(2):
        rows = st.U[:, d, :2, :].reshape(ns, 6)
        f[12 * d + 0:12 * d + 12:2] = rows.real.T
        f[12 * d + 1:12 * d + 12:2] = rows.imag.T
    f[24:32] = st.E[:, 0].T
    f[32:40] = st.E[:, 1].T
    f[40:48] = st.phi.T
    f[48:56] = st.pi.T
    g = f.reshape(7, 8, ns).transpose(0, 2, 1).reshape(-1)  # plane p, site s -> ((p//8) ns + s) 8 + p%8
    return torch.tensor(g.astype(np.float32 if prec else np.float64), device="cuda").contiguous()


def call(buf_ptr, n, prec, tau, expanding=1):
    out = np.zeros(8)
    rc = G.lib().glasma_diagnostics_noalloc(C.c_void_p(buf_ptr), n, prec, expanding, tau, None,
                                            out.ctypes.data_as(C.c_void_p))
    return rc, out


def tiled_state(small, n):
    """A periodic n x n state repeating a small periodic state (n a multiple of its size)."""
    m = small.n
    X, Y = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    idx = ((X % m) + m * (Y % m)).reshape(-1)
    st = type(small)(n, step=small.step)
    st.U[...] = small.U[idx]
    st.E[...] = small.E[idx]
    st.phi[...] = small.phi[idx]
    st.pi[...] = small.pi[idx]
    return st


@pytest.mark.parametrize("prec,n,tol,expanding", [(0, 24, 1e-12, 1), (1, 40, 2e-5, 1), (0, 67, 1e-12, 1),
                                                  (0, 30, 1e-12, 0), (1, 33, 2e-5, 0), (1, 1024, 2e-5, 1)])
def test_noalloc_diagnostics_match_context_diagnostics(prec, n, tol, expanding):
    # n = 1024: the largest lattice the static scratch takes (4096 blocks, the last partials
    # right before the slot of the final sums)
    st = random_state(n, seed=500 + n, step=5) if n <= 67 else tiled_state(random_state(32, seed=532, step=5), n)
    g = G.Glasma(n, 6.0, precision=prec, tau_end_fm=100.0, expanding=expanding)
    g.set_state(st.U, st.E, st.phi, st.pi, st.step)
    want = g.diagnostics()
    buf = plane_buffer(st, prec)
    torch.cuda.synchronize()
    for _ in range(2):  # the static scratch keeps the previous call's contents
        rc, got = call(buf.data_ptr(), n, prec, st.step * 0.125, expanding)
        assert rc == 0
        assert abs(got[0] - want[0]) <= tol * max(want[0], 1e-300) + 1e-15
        assert rel_err(got[1:5], want[1:5]) < tol
        assert abs(got[5] - want[5]) <= tol + 1e-15
        assert got[6] == want[6] and got[7] == want[7] == 0


def test_noalloc_rejects_lattices_beyond_the_scratch():
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    rc, _ = call(buf.data_ptr(), 1025, 1, 1.0)
    assert rc == -1
    assert b"static scratch" in G.lib().glasma_last_error()


def test_noalloc_rejects_unaligned_buffers():
    buf = torch.zeros(4 * 56 * 64 + 4, dtype=torch.float32, device="cuda")
    rc = G.lib().glasma_diagnostics_noalloc(C.c_void_p(buf.data_ptr() + 4), 8, 1, 1, 1.0, None,
                                            np.zeros(8).ctypes.data_as(C.c_void_p))
    assert rc == -1
    assert b"aligned" in G.lib().glasma_last_error()


def test_noalloc_rejects_host_memory_and_bad_tau():
    host = np.zeros(56 * 64, dtype=np.float32)
    rc, _ = call(host.ctypes.data, 8, 1, 1.0)
    assert rc == -1
    assert b"device memory" in G.lib().glasma_last_error()
    buf = torch.zeros(56 * 64, dtype=torch.float32, device="cuda")
    rc, _ = call(buf.data_ptr(), 8, 1, 0.0, expanding=1)
    assert rc == -1
    assert b"tau > 0" in G.lib().glasma_last_error()


def test_noalloc_refuses_a_capturing_stream():
    buf = torch.zeros(56 * 64, dtype=torch.float32, device="cuda")
    s = torch.cuda.Stream()
    out = np.zeros(8)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    rc = None
    with torch.cuda.graph(g, stream=s, capture_error_mode="relaxed"):
        rc = G.lib().glasma_diagnostics_noalloc(C.c_void_p(buf.data_ptr()), 8, 1, 1, 1.0, C.c_void_p(s.cuda_stream),
                                                out.ctypes.data_as(C.c_void_p))
    assert rc == -1
    assert b"captured" in G.lib().glasma_last_error()
