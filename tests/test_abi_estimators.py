"""broadening_transport (the library's Eq. 3 estimator, host code behind the C ABI) against
the oracle's o_transport_coefficients, and the oracle's pins applied to the library.
No device work: runs without a GPU."""
import ctypes as C

import numpy as np
import pytest

import oracle as O
from test_oracle_estimators import pin_failures

L = pytest.importorskip("paper_2307_07999_gb300._lib")

INVALID = -1


@pytest.fixture(scope="module")
def lib():
    from paper_2307_07999_gb300 import build

    build.build()
    return L.lib()


def _call(lib, tab, kind):
    tab = np.ascontiguousarray(tab, dtype=np.float64)
    out = np.zeros((tab.shape[0], 8))
    rc = lib.broadening_transport(tab.ctypes.data_as(C.c_void_p), tab.shape[0], tab.shape[1], kind,
                                  out.ctypes.data_as(C.c_void_p))
    return rc, out


def test_library_meets_the_oracle_pins(lib):
    def est(tab, kind):
        rc, out = _call(lib, tab, L.GLASMA_HEAVY_QUARKS if kind == "hq" else L.GLASMA_JETS_X)
        assert rc == 0
        return out

    assert pin_failures(est) == []


@pytest.mark.parametrize("rows", [1, 2, 3, 17, 410])
@pytest.mark.parametrize("kind", ["hq", "jet"])
def test_library_equals_oracle_on_random_tables(lib, rows, kind):
    rng = np.random.default_rng(rows)
    tab = np.zeros((rows, 5))
    tab[:, 0] = np.cumsum(rng.uniform(0.001, 0.01, rows))
    tab[:, 1:4] = rng.normal(size=(rows, 3))
    tab[:, 4] = 1e4
    rc, got = _call(lib, tab, L.GLASMA_HEAVY_QUARKS if kind == "hq" else L.GLASMA_JETS_X)
    assert rc == 0
    want = O.transport_coefficients(tab, kind)
    assert np.allclose(got, want, rtol=1e-14, atol=1e-14, equal_nan=True)


def test_wider_rows_are_read_by_stride(lib):
    rng = np.random.default_rng(3)
    tab = np.zeros((30, 7))
    tab[:, 0] = np.linspace(0.05, 1.0, 30)
    tab[:, 1:7] = rng.normal(size=(30, 6))
    rc, got = _call(lib, tab, L.GLASMA_HEAVY_QUARKS)
    assert rc == 0
    assert np.allclose(got, O.transport_coefficients(tab[:, :5]), rtol=1e-14, atol=1e-14, equal_nan=True)


def test_bad_arguments_are_rejected(lib):
    tab = np.zeros((4, 5))
    tab[:, 0] = [0.1, 0.2, 0.2, 0.3]  # tau does not increase
    rc, _ = _call(lib, tab, L.GLASMA_HEAVY_QUARKS)
    assert rc == INVALID and lib.glasma_last_error()
    tab[:, 0] = [0.1, 0.2, 0.3, 0.4]
    assert _call(lib, tab, 7)[0] == INVALID
    out = np.zeros((4, 8))
    assert lib.broadening_transport(tab.ctypes.data_as(C.c_void_p), 4, 3, 0, out.ctypes.data_as(C.c_void_p)) == INVALID
    assert lib.broadening_transport(None, 4, 5, 0, out.ctypes.data_as(C.c_void_p)) == INVALID
    assert lib.broadening_transport(tab.ctypes.data_as(C.c_void_p), 0, 5, 0, out.ctypes.data_as(C.c_void_p)) == INVALID


def test_binding_marshals_only():
    import paper_2307_07999_gb300 as G

    rng = np.random.default_rng(9)
    tab = np.zeros((12, 5))
    tab[:, 0] = np.linspace(0.1, 1.2, 12)
    tab[:, 1:4] = rng.normal(size=(12, 3))
    assert np.array_equal(G.kappa_qhat(tab), G.broadening_transport(tab)[:, :4])
    assert np.array_equal(G.anisotropy(tab, "jet"), G.broadening_transport(tab, "jet")[:, [0, 7]], equal_nan=True)
