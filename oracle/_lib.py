"""Build and load the oracle's C library (test infrastructure only).

The shared object is compiled with the system C compiler from
``schur_oracle.c`` next to this file, with ``-ffp-contract=off`` so every
rounding is the one written in the source.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "schur_oracle.c")
_SO = os.path.join(_HERE, "_schur_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle library if it is missing or older than its source."""
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    cc = os.environ.get("CC", "gcc")
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = [cc, "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_SO)
        _declare(_lib)
    return _lib


_P = ctypes.c_void_p
_I = ctypes.c_int


def _declare(L):
    L.sro_alg2_f64.argtypes = [_I, _P, _I, _P, _I, _P, _P, _I, ctypes.c_double, _I]
    L.sro_alg2_f32.argtypes = [_I, _P, _I, _P, _I, _P, _P, _I, ctypes.c_double, _I]
    L.sro_alg2_c128.argtypes = [_I, _P, _I, _P, _I, _P, _P, _I, ctypes.c_double, _I]
    L.sro_alg2_c64.argtypes = [_I, _P, _I, _P, _I, _P, _P, _I, ctypes.c_double, _I]
    L.sro_alg3_f64.argtypes = [_I, _P, _I, _P, _I, _P, _I, _I]
    L.sro_kron_solve.argtypes = [_I, _P, _I, _P, _I, _P, _P, _I]
    L.sro_gemm_dd.argtypes = [_I, _I, _I, _I, _P, _P, _I, _P, _P, _I, _P, _P, _I]
    L.sro_gemm_dd.restype = None
    L.sro_residuals_dd.argtypes = [_I, _P, _I, _P, _I, _P, _P]
    L.sro_residuals_dd.restype = None
    L.sro_residuals_dd_quasi.argtypes = [_I, _P, _I, _P, _I, _P, _P, _P]
    L.sro_residuals_dd_quasi.restype = None
    L.sro_residuals_dd_c.argtypes = [_I, _P, _I, _P, _I, _P, _P]
    L.sro_residuals_dd_c.restype = None
    L.sro_sample_entries_dd.argtypes = [_I, _P, _I, _P, _I, _I, _P, _P, _P, _P]
    L.sro_sample_entries_dd.restype = None
    L.sro_sample_entries_dd_c.argtypes = [_I, _P, _I, _P, _I, _I, _P, _P, _P, _P]
    L.sro_sample_entries_dd_c.restype = None
    L.sro_alg2_f64_dd.argtypes = [_I, _P, _I, _P, _I, _P, _P, _P, _I, ctypes.c_double]
    L.sro_alg2_f64_dd.restype = ctypes.c_int
    L.sro_residuals_q.argtypes = [_I, _P, _P, _I, _P, _P, _I, _P, _P]
    L.sro_residuals_q.restype = None
    L.sro_sample_entries_q.argtypes = [_I, _P, _P, _I, _P, _P, _I, _I, _P, _P, _P, _P, _P, _P]
    L.sro_sample_entries_q.restype = None
    for name in ("sro_alg2_quasi_f64", "sro_alg2_quasi_f32"):
        getattr(L, name).argtypes = [_I, _P, _I, _P, _I, _P, _P, _P, _I, ctypes.c_double]
        getattr(L, name).restype = ctypes.c_int
    L.sro_set_threads.argtypes = [_I]
    L.sro_set_threads.restype = None
    L.sro_max_threads.argtypes = []
    L.sro_max_threads.restype = ctypes.c_int
    for name in ("sro_alg2_f64", "sro_alg2_f32", "sro_alg2_c128", "sro_alg2_c64",
                 "sro_alg3_f64", "sro_kron_solve"):
        getattr(L, name).restype = ctypes.c_int


def ptr(a: np.ndarray) -> ctypes.c_void_p:
    return ctypes.c_void_p(a.ctypes.data)


def fortran(a: np.ndarray, dtype) -> np.ndarray:
    return np.asfortranarray(np.asarray(a, dtype=dtype))


def set_threads(n: int) -> None:
    """Thread count of the oracle's OpenMP loops."""
    lib().sro_set_threads(int(n))


def max_threads() -> int:
    return int(lib().sro_max_threads())


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
