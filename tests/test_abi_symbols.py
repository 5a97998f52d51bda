"""The C-ABI library loads without a GPU and exports every function that
include/glasma.h declares (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "glasma.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("glasma_init", "glasma_step", "cpic_init", "cpic_push", "broadening_accumulate"):
        assert required in names


def test_library_exports_all_declared_symbols():
    from paper_2307_07999_gb300 import build

    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_has_no_cpu_fallback():
    import paper_2307_07999_gb300._lib as L

    for name in L.SIGNATURES:
        assert name in declared_functions()
