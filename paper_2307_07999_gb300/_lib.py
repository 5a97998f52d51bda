"""ctypes declarations of the C ABI in include/glasma.h."""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libglasma.so")

GLASMA_FP64 = 0
GLASMA_FP32 = 1

GLASMA_HEAVY_QUARKS = 0
GLASMA_JETS_X = 1

GLASMA_BATCH_GRAPH = 0
GLASMA_BATCH_PERSISTENT = 1
GLASMA_BATCH_PER_EVENT = 2
GLASMA_BATCH_EAGER = 3

STATUS = {
    0: "GLASMA_OK",
    -1: "GLASMA_ERR_INVALID",
    -2: "GLASMA_ERR_CUDA",
    -3: "GLASMA_ERR_NONFINITE",
    -4: "GLASMA_ERR_TIMEOUT",
    -5: "GLASMA_ERR_NOCONV",
    -6: "GLASMA_ERR_NOSPACE",
}


class GlasmaError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class GlasmaParams(C.Structure):
    _fields_ = [
        ("n", C.c_int32),
        ("n_sheets", C.c_int32),
        ("L_fm", C.c_double),
        ("g2mu_GeV", C.c_double),
        ("m_ir_GeV", C.c_double),
        ("dtau_over_a", C.c_double),
        ("tau_end_fm", C.c_double),
        ("precision", C.c_int32),
        ("reunit_every", C.c_int32),
        ("expanding", C.c_int32),
        ("newton_max_iter", C.c_int32),
        ("newton_tol", C.c_double),
        ("seed", C.c_uint64),
    ]


class CorrParams(C.Structure):
    _fields_ = [("tau_start_fm", C.c_double), ("ox0", C.c_double)]


class CpicParams(C.Structure):
    _fields_ = [
        ("n_particles", C.c_int32),
        ("init_kind", C.c_int32),
        ("mass_GeV", C.c_double),
        ("tau_form_fm", C.c_double),
        ("p_min_GeV", C.c_double),
        ("p_max_GeV", C.c_double),
        ("q2", C.c_double),
        ("q3", C.c_double),
        ("bin_every", C.c_int32),
        ("integrator", C.c_int32),
        ("substeps", C.c_int32),
        ("interp", C.c_int32),
        ("seed", C.c_uint64),
    ]


_p = C.c_void_p
_i32 = C.c_int32
_i64 = C.c_int64
_d = C.c_double
_pp = C.POINTER(C.c_void_p)

SIGNATURES = {
    "glasma_workspace_bytes": (_i64, [C.POINTER(GlasmaParams)]),
    "glasma_create": (C.c_int, [C.POINTER(GlasmaParams), _p, _i64, _p, _pp]),
    "glasma_init": (C.c_int, [_p]),
    "glasma_ic_stats": (C.c_int, [_p, C.POINTER(_i64), C.POINTER(_d), C.POINTER(_i32)]),
    "glasma_init_from_host": (C.c_int, [_p, _p, _p, _p, _p, _i32]),
    "glasma_get_state": (C.c_int, [_p, _p, _p, _p, _p, C.POINTER(_i32)]),
    "glasma_step": (C.c_int, [_p, _i32]),
    "glasma_diagnostics": (C.c_int, [_p, _p]),
    "glasma_destroy": (None, [_p]),
    "cpic_workspace_bytes": (_i64, [C.POINTER(GlasmaParams), C.POINTER(CpicParams)]),
    "cpic_create": (C.c_int, [_p, C.POINTER(CpicParams), _p, _i64, _pp]),
    "cpic_init": (C.c_int, [_p]),
    "cpic_init_from_host": (C.c_int, [_p] + [_p] * 8),
    "cpic_get_particles": (C.c_int, [_p] + [_p] * 7),
    "cpic_push": (C.c_int, [_p, _i32]),
    "cpic_push_many": (C.c_int, [_p, _i32, _i32]),
    "glasma_batch_set_graph_timing": (C.c_int, [_p, _i32]),
    "glasma_batch_set_push_stream": (C.c_int, [_p, _i32]),
    "glasma_batch_set_wait_limit": (C.c_int, [_p, _i64]),
    "glasma_batch_graph_times": (C.c_int, [_p, C.POINTER(_d), C.POINTER(_i64), C.POINTER(_d)]),
    "glasma_state_bytes": (_i64, [_p]),
    "glasma_export_state": (C.c_int, [_p, _p, _i64]),
    "glasma_import_state": (C.c_int, [_p, _p, _i64]),
    "cpic_state_bytes": (_i64, [_p]),
    "cpic_export_state": (C.c_int, [_p, _p, _i64]),
    "cpic_import_state": (C.c_int, [_p, _p, _i64]),
    "broadening_accumulate": (C.c_int, [_p, _p, _i64, C.POINTER(_i64)]),
    "broadening_transport": (C.c_int, [_p, _i64, _i32, _i32, _p]),
    "cpic_casimir_drift": (C.c_int, [_p, _p]),
    "cpic_destroy": (None, [_p]),
    "glasma_batch_workspace_bytes": (_i64, [C.POINTER(GlasmaParams), C.POINTER(CpicParams), _i32]),
    "glasma_batch_create": (C.c_int, [C.POINTER(GlasmaParams), C.POINTER(CpicParams), _i32, _p, _i64, _p, _pp]),
    "glasma_batch_init": (C.c_int, [_p, C.POINTER(_i64)]),
    "glasma_batch_run": (C.c_int, [_p, _i32]),
    "glasma_batch_work": (C.c_int, [_p, C.POINTER(_i64), C.POINTER(_i64)]),
    "glasma_batch_broadening": (C.c_int, [_p, _i32, _p, _i64, C.POINTER(_i64)]),
    "glasma_batch_diagnostics": (C.c_int, [_p, _i32, _p]),
    "glasma_batch_state_bytes": (_i64, [_p]),
    "glasma_batch_export_state": (C.c_int, [_p, _p, _i64]),
    "glasma_batch_import_state": (C.c_int, [_p, _p, _i64]),
    "glasma_batch_profile": (C.c_int, [_p, _i32, C.POINTER(_d), C.POINTER(_i64), C.POINTER(_i64), C.POINTER(_i64),
                                       C.POINTER(_d)]),
    "glasma_batch_launches": (_i64, [_p, _i32]),
    "glasma_field_tile_variants": (_i32, [_i32]),
    "glasma_field_tile_shape": (C.c_int, [_i32, _i32, C.POINTER(_i32), C.POINTER(_i32), C.POINTER(_i32)]),
    "glasma_batch_variant": (_i32, [_p]),
    "glasma_batch_set_variant": (C.c_int, [_p, _i32]),
    "glasma_batch_tune": (C.c_int, [_p, _i32, C.POINTER(_i32), C.POINTER(_d)]),
    "glasma_push_variants": (_i32, []),
    "corr_workspace_bytes": (_i64, [_p]),
    "corr_create": (C.c_int, [_p, _p, _p, _i64, C.POINTER(_p)]),
    "corr_table": (C.c_int, [_p, _p, _i64, C.POINTER(_i64)]),
    "corr_destroy": (None, [_p]),
    "glasma_batch_push_variant": (_i32, [_p]),
    "glasma_batch_set_push_variant": (C.c_int, [_p, _i32]),
    "glasma_batch_get_particles": (C.c_int, [_p, _i32] + [_p] * 7),
    "glasma_batch_destroy": (None, [_p]),
    "glasma_diagnostics_noalloc": (C.c_int, [_p, _i32, _i32, _i32, _d, _p, _p]),
    "glasma_mlp_workspace_bytes": (_i64, []),
    "glasma_mlp_create": (C.c_int, [_p, _i64, C.c_uint64, _p, _pp]),
    "glasma_mlp_destroy": (None, [_p]),
    "glasma_mlp_set_scales": (C.c_int, [_p, C.c_float, C.c_float]),
    "glasma_mlp_fit_scales": (C.c_int, [_p, _p, _p, _i64]),
    "glasma_mlp_train": (C.c_int, [_p, _p, _p, _i64, _i32, _i32, C.c_float, C.POINTER(_d)]),
    "glasma_mlp_loss_grad": (C.c_int, [_p, _p, _p, _i64, C.POINTER(_d), _p]),
    "glasma_mlp_predict": (C.c_int, [_p, _p, _i64, _p]),
    "glasma_mlp_get_params": (C.c_int, [_p, _p, _p]),
    "glasma_mlp_set_params": (C.c_int, [_p, _p]),
    "glasma_ic_dataset": (C.c_int, [_p, _p, _p]),
    "glasma_init_warm": (C.c_int, [_p, _p]),
    "glasma_last_error": (C.c_char_p, []),
}

_LIB = None


def lib():
    """The loaded libglasma.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"{LIB_PATH} is missing: build it with `python -c \"import __graft_entry__ as g; g.build()\"`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def check(status):
    if status != 0:
        raise GlasmaError(status, lib().glasma_last_error().decode())
    return status
