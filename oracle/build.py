"""Builds the FP64 CPU oracle into oracle/liboracle.so with gcc.

Test infrastructure only (see oracle.h): imported by tests/, by
__graft_entry__ (build + smoke) and by bench.py's CPU-baseline leg.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["su3.c", "philox.c", "fft.c", "ic.c", "field.c", "particles.c", "correlators.c", "estimators.c", "mlp.c"]
LIB = os.path.join(HERE, "liboracle.so")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = SOURCES + ["oracle.h"]
    return any(os.path.getmtime(os.path.join(HERE, f)) > t for f in deps
               if os.path.exists(os.path.join(HERE, f)))


def build(force: bool = False, openmp: bool = True) -> str:
    if not force and not _stale():
        return LIB
    srcs = [os.path.join(HERE, f) for f in SOURCES if os.path.exists(os.path.join(HERE, f))]
    base = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-o", LIB + ".tmp"] + srcs + ["-lm"]
    cmd = base[:1] + (["-fopenmp"] if openmp else []) + base[1:]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and openmp:
        r = subprocess.run(base, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("oracle build failed:\n" + r.stderr)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
