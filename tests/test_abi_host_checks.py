"""Argument checks of the C ABI that run on the host before any device work: the
library rejects bad parameters with GLASMA_ERR_INVALID and a message, and reports its
compiled variants, all without a GPU."""
import ctypes as C

import pytest

L = pytest.importorskip("paper_2307_07999_gb300._lib")
W = pytest.importorskip("paper_2307_07999_gb300.workloads")

INVALID = -1


@pytest.fixture(scope="module")
def lib():
    from paper_2307_07999_gb300 import build

    build.build()
    return L.lib()


def params(**kw):
    p = W.glasma_params(64, 6.0, 2.0, 1, L.GLASMA_FP32)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@pytest.mark.parametrize("bad", [dict(n=1), dict(n=20000), dict(L_fm=0.0), dict(dtau_over_a=0.0),
                                 dict(dtau_over_a=1.5), dict(precision=7), dict(n_sheets=0), dict(tau_end_fm=-1.0)])
def test_field_parameters_are_checked(lib, bad):
    assert lib.glasma_workspace_bytes(C.byref(params(**bad))) == INVALID
    assert lib.glasma_last_error()


def test_particle_parameters_are_checked(lib):
    gp = params()
    for bad in (dict(n_particles=-1), dict(mass_GeV=-1.0), dict(init_kind=5), dict(p_min_GeV=3.0, p_max_GeV=1.0),
                dict(integrator=2), dict(integrator=-1), dict(substeps=-1), dict(substeps=65), dict(interp=2)):
        pp = W.charm_params(10, 1)
        for k, v in bad.items():
            setattr(pp, k, v)
        assert lib.cpic_workspace_bytes(C.byref(gp), C.byref(pp)) == INVALID, bad


def test_batch_event_lists_are_checked(lib):
    evs = (L.GlasmaParams * 2)(params(), params(precision=L.GLASMA_FP64))  # mixed precision
    pps = (L.CpicParams * 2)(W.charm_params(10, 1), W.charm_params(10, 2))
    assert lib.glasma_batch_workspace_bytes(evs, pps, 2) == INVALID
    assert b"precision" in lib.glasma_last_error()
    assert lib.glasma_batch_workspace_bytes(evs, pps, 0) == INVALID
    one = (L.GlasmaParams * 1)(params())
    pone = (L.CpicParams * 1)(W.charm_params(10, 1))
    h = C.c_void_p()
    # workspace not 256-byte aligned, or null
    assert lib.glasma_batch_create(one, pone, 1, C.c_void_p(16), 1 << 20, None, C.byref(h)) == INVALID
    assert lib.glasma_batch_create(one, pone, 1, None, 1 << 20, None, C.byref(h)) == INVALID


def test_compiled_variants_are_reported(lib):
    nv = lib.glasma_field_tile_variants(L.GLASMA_FP32)
    assert nv >= 8 and lib.glasma_field_tile_variants(L.GLASMA_FP64) == 1
    a, b, c = C.c_int32(), C.c_int32(), C.c_int32()
    assert lib.glasma_field_tile_shape(L.GLASMA_FP32, 0, C.byref(a), C.byref(b), C.byref(c)) == 0
    assert (a.value, b.value, c.value) == (32, 4, 3)
    shapes = set()
    for v in range(nv):
        assert lib.glasma_field_tile_shape(L.GLASMA_FP32, v, C.byref(a), C.byref(b), C.byref(c)) == 0
        assert a.value * b.value % 32 == 0 and 1 <= c.value <= 8
        shapes.add((a.value, b.value, c.value))
    assert len(shapes) == nv
    assert lib.glasma_field_tile_shape(L.GLASMA_FP32, nv, C.byref(a), C.byref(b), C.byref(c)) == INVALID
    assert lib.glasma_push_variants() == 4  # fields through L1, staged, record, split


def test_network_and_monitor_entry_points_check_their_buffers(lib):
    assert lib.glasma_mlp_workspace_bytes() > 23312 * 4
    h = C.c_void_p()
    assert lib.glasma_mlp_create(C.c_void_p(8), 1 << 24, 1, None, C.byref(h)) == INVALID  # misaligned
    out = (C.c_double * 8)()
    assert lib.glasma_diagnostics_noalloc(None, 8, 1, 1, 1.0, None, out) == INVALID
    assert lib.glasma_diagnostics_noalloc(C.c_void_p(256), 4096, 1, 1, 1.0, None, out) == INVALID  # > scratch
    assert b"static scratch" in lib.glasma_last_error()
