"""The C-ABI library loads, exports every declared symbol and validates its
arguments on the host (no GPU needed: these calls return before any CUDA call)."""
import ctypes
import glob
import os
import re

import pytest

from paper_2203_10879_gb300 import _binding as B
from paper_2203_10879_gb300 import build as build_mod

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build_mod.build()
    return B.lib()


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(schur_refine_\w+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported(L):
    declared = _declared()
    assert declared, "no declarations found"
    for name in declared:
        assert hasattr(L, name), name
    assert set(B.EXPORTS) == declared


def test_default_options(L):
    o = B.default_options()
    assert (o.dtype, o.hp_gemm, o.lp, o.qhat_type, o.full_sigma, o.max_iter) == (0, 0, 0, 0, 0, 10)
    assert (o.batch_mode, o.tune, o.graph, o.solve_mode, o.symmetric, o.l_cap) == (0, 0, 0, 0, 0, 0.0)
    # the binding's struct has the C struct's size (the library fills every field)
    raw = (ctypes.c_char * (ctypes.sizeof(B.sr_options) + 64))(*([b"\xab"] * (ctypes.sizeof(B.sr_options) + 64)))
    L.schur_refine_default_options(ctypes.cast(raw, ctypes.POINTER(B.sr_options)))
    assert bytes(raw[ctypes.sizeof(B.sr_options):]) == b"\xab" * 64


def test_null_handle_and_bad_arguments(L):
    P = ctypes.c_void_p
    assert L.schur_refine_step(None, 4, P(1), 4, P(1), 4, None, None, None) == B.SR_ERR_INVALID_ARG
    assert L.schur_refine_residuals(None, 4, P(1), 4, P(1), 4, None, None) == B.SR_ERR_INVALID_ARG
    assert L.schur_refine_trisolve(None, 4, P(1), 4, P(1)) == B.SR_ERR_INVALID_ARG
    assert L.schur_refine_selftest_wait_timeout(None) == B.SR_ERR_INVALID_ARG
    assert L.schur_refine_gemm(None, 0, 4, 4, 4, P(1), 4, P(1), 4, P(1), 4) == B.SR_ERR_INVALID_ARG
    assert L.schur_refine_batched(None, 1, None, None, None, None, None, None) == B.SR_ERR_INVALID_ARG
    p = B.sr_profile()
    assert L.schur_refine_get_profile(None, ctypes.byref(p)) == B.SR_ERR_INVALID_ARG
    L.schur_refine_destroy(None)


def test_create_rejects_bad_sizes_and_options(L):
    h = ctypes.c_void_p(123)
    assert L.schur_refine_create(ctypes.byref(h), 0, None, None) == B.SR_ERR_INVALID_ARG
    assert h.value is None
    o = B.default_options(lp=7)
    assert L.schur_refine_create(ctypes.byref(h), 8, ctypes.byref(o), None) == B.SR_ERR_INVALID_ARG
    o = B.default_options(hp_gemm=9)
    assert L.schur_refine_create(ctypes.byref(h), 8, ctypes.byref(o), None) == B.SR_ERR_INVALID_ARG
    o = B.default_options(ozaki_slices=99)
    assert L.schur_refine_create(ctypes.byref(h), 8, ctypes.byref(o), None) == B.SR_ERR_INVALID_ARG
    for bad in ({"solve_mode": 3}, {"solve_mode": -1}, {"graph": 2}, {"tune": 2}, {"batch_mode": 5},
                {"symmetric": 2}, {"l_cap": -1.0}, {"l_cap": float("nan")}, {"l_cap": float("inf")}):
        o = B.default_options(**bad)
        assert L.schur_refine_create(ctypes.byref(h), 8, ctypes.byref(o), None) == B.SR_ERR_INVALID_ARG, bad
        assert h.value is None
    assert L.schur_refine_create(None, 8, None, None) == B.SR_ERR_INVALID_ARG


def test_status_strings(L):
    for s in range(9):
        assert B.status_string(s)
    assert "distinct" in B.status_string(B.SR_ERR_NONDISTINCT)


def test_binding_refuses_host_tensors():
    torch = pytest.importorskip("torch")
    with pytest.raises(ValueError):
        B._dev(torch.zeros(4, 4), "A")
