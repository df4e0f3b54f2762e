"""ctypes binding of libschur_refine.so (argument marshalling only).

Each function has the name of the C entry point it calls and takes device
buffers as torch tensors laid out column-major (``t.stride(0) == 1``; a
Fortran-ordered numpy array moved with ``torch.from_numpy(a).cuda()`` keeps
that layout only if copied with ``colmajor``). Every step of the iteration runs
in the CUDA library; nothing here computes. If the shared library has not been
built, every call raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libschur_refine.so")

SR_OK, SR_ERR_INVALID_ARG, SR_ERR_NONDISTINCT, SR_ERR_NONFINITE = 0, 1, 2, 3
SR_ERR_NOT_CONVERGED, SR_ERR_TIMEOUT, SR_ERR_CUDA, SR_ERR_OOM, SR_ERR_UNSUPPORTED = 4, 5, 6, 7, 8
SR_REAL, SR_COMPLEX = 0, 1
SR_TARGET_FP64, SR_TARGET_DD, SR_TARGET_TD, SR_TARGET_D6 = 0, 1, 2, 3
SR_HP_FP64, SR_HP_OZAKI_BF16, SR_HP_OZAKI_CRT = 0, 1, 2
SR_LP_FP32, SR_LP_FP64 = 0, 1
SR_QHAT_FP32, SR_QHAT_FP64 = 0, 1
PROF_KINDS = 8
PROF_NAMES = ["hp_gemm", "oz_split", "oz_mma", "oz_combine", "solve", "lp_gemm", "other", "spare"]

#: every symbol include/schur_refine.h declares
EXPORTS = [
    "schur_refine_default_options", "schur_refine_create", "schur_refine_step",
    "schur_refine_batched", "schur_refine_residuals", "schur_refine_trisolve",
    "schur_refine_gemm", "schur_refine_get_profile", "schur_refine_reset_profile",
    "schur_refine_destroy", "schur_refine_status_string", "schur_refine_residuals_noalloc",
    "schur_refine_selftest_wait_timeout", "schur_refine_solve_plan", "schur_refine_crt_info",
]


class sr_options(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int), ("target", ctypes.c_int), ("hp_gemm", ctypes.c_int),
                ("lp", ctypes.c_int), ("qhat_type", ctypes.c_int), ("full_sigma", ctypes.c_int),
                ("max_iter", ctypes.c_int), ("ozaki_slices", ctypes.c_int), ("tol", ctypes.c_double),
                ("profile", ctypes.c_int), ("batch_streams", ctypes.c_int), ("batch_mode", ctypes.c_int),
                ("tune", ctypes.c_int), ("graph", ctypes.c_int), ("solve_mode", ctypes.c_int),
                ("symmetric", ctypes.c_int), ("l_cap", ctypes.c_double), ("lp_slices", ctypes.c_int),
                ("quasi", ctypes.c_int)]


class sr_norms(ctypes.Structure):
    _fields_ = [("stril_rel", ctypes.c_double), ("orth", ctypes.c_double), ("w_norm", ctypes.c_double),
                ("iters", ctypes.c_int), ("hp_gemms", ctypes.c_int)]


class sr_profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * PROF_KINDS), ("flops", ctypes.c_longlong * PROF_KINDS),
                ("bytes", ctypes.c_longlong * PROF_KINDS), ("launches", ctypes.c_longlong * PROF_KINDS),
                ("spans", ctypes.c_longlong * PROF_KINDS)]

    def as_dict(self):
        return {name: {"ms": self.ms[k], "flops": self.flops[k], "bytes": self.bytes[k],
                       "launches": self.launches[k], "spans": self.spans[k]}
                for k, name in enumerate(PROF_NAMES)}


class SchurRefineError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        super().__init__(f"{what}: {status_string(status)} ({status})")
        self.status = status


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded CUDA library; raises if it was not built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(the refinement has no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.schur_refine_default_options.argtypes = [ctypes.POINTER(sr_options)]
        L.schur_refine_default_options.restype = None
        L.schur_refine_create.argtypes = [ctypes.POINTER(P), I, ctypes.POINTER(sr_options), P]
        L.schur_refine_step.argtypes = [P, I, P, I, P, I, P, P, ctypes.POINTER(sr_norms)]
        L.schur_refine_batched.argtypes = [P, I, ctypes.POINTER(I), ctypes.POINTER(P), ctypes.POINTER(P),
                                           ctypes.POINTER(P), ctypes.POINTER(I), ctypes.POINTER(I)]
        L.schur_refine_residuals.argtypes = [P, I, P, I, P, I, ctypes.POINTER(D), ctypes.POINTER(D)]
        L.schur_refine_residuals_noalloc.argtypes = [I, P, I, P, I, ctypes.POINTER(D), ctypes.POINTER(D), P]
        L.schur_refine_trisolve.argtypes = [P, I, P, I, P]
        L.schur_refine_selftest_wait_timeout.argtypes = [P]
        L.schur_refine_solve_plan.argtypes = [I, ctypes.POINTER(ctypes.c_ulonglong), ctypes.c_longlong,
                                              ctypes.POINTER(ctypes.c_longlong)]
        L.schur_refine_gemm.argtypes = [P, I, I, I, I, P, I, P, I, P, I]
        L.schur_refine_crt_info.argtypes = [I, I, ctypes.c_longlong, ctypes.POINTER(I), ctypes.POINTER(ctypes.c_uint),
                                            ctypes.POINTER(ctypes.c_uint), ctypes.POINTER(I), ctypes.POINTER(I)]
        L.schur_refine_get_profile.argtypes = [P, ctypes.POINTER(sr_profile)]
        L.schur_refine_reset_profile.argtypes = [P]
        L.schur_refine_destroy.argtypes = [P]
        L.schur_refine_destroy.restype = None
        L.schur_refine_status_string.argtypes = [I]
        L.schur_refine_status_string.restype = ctypes.c_char_p
        for f in ("schur_refine_create", "schur_refine_step", "schur_refine_batched",
                  "schur_refine_residuals", "schur_refine_trisolve", "schur_refine_gemm",
                  "schur_refine_get_profile", "schur_refine_reset_profile",
                  "schur_refine_residuals_noalloc", "schur_refine_selftest_wait_timeout",
                  "schur_refine_solve_plan", "schur_refine_crt_info"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


def status_string(status: int) -> str:
    return lib().schur_refine_status_string(int(status)).decode()


# ---- marshalling helpers -------------------------------------------------------

def _dev(t, what):
    """(pointer, leading dimension) of a column-major CUDA tensor, or (None, 0)."""
    if t is None:
        return None, 0
    if isinstance(t, int):
        return t, 0
    if not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor")
    if t.dim() == 1:
        return t.data_ptr(), t.shape[0]
    if t.stride(0) != 1 and t.shape[0] > 1:
        raise ValueError(f"{what} must be column-major (stride(0) == 1)")
    ld = t.stride(1) if t.shape[1] > 1 else t.shape[0]
    return t.data_ptr(), max(ld, t.shape[0])


def colmajor(t):
    """A column-major copy of a 2-D tensor (same device and dtype)."""
    return t.t().contiguous().t()


def dd_pair(t):
    """(hi, lo) views of a double-double matrix held as one column-major
    tensor of shape (n, 2c): the hi plane in columns [0, c), lo in [c, 2c) --
    the layout the C ABI expects for SR_TARGET_DD (lo plane ld * c elements
    after hi)."""
    c = t.shape[1] // 2
    return t[:, :c], t[:, c:]


def default_options(**kw) -> sr_options:
    o = sr_options()
    lib().schur_refine_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


# ---- the C entry points ------------------------------------------------------------

def schur_refine_create(n_max: int, opt: sr_options | None = None, stream=None):
    """Returns (status, handle)."""
    h = ctypes.c_void_p()
    st = ctypes.c_void_p(int(stream)) if stream is not None else None
    s = lib().schur_refine_create(ctypes.byref(h), int(n_max), ctypes.byref(opt) if opt is not None else None, st)
    return s, h


def schur_refine_step(h, n: int, A, Q, Qhat=None, T=None):
    """Returns (status, sr_norms)."""
    pa, lda = _dev(A, "A")
    pq, ldq = _dev(Q, "Q")
    ph, ldh = _dev(Qhat, "Qhat")
    pt, _ = _dev(T, "T")
    if ph is not None and ldh and ldh != ldq:
        raise ValueError("Qhat must have the leading dimension of Q")
    out = sr_norms()
    s = lib().schur_refine_step(h, int(n), pa, lda, pq, ldq, ph, pt, ctypes.byref(out))
    return s, out


def schur_refine_batched(h, ns, As, Qs, Qhats=None):
    """Returns (status, iters list, status list)."""
    b = len(ns)
    N = (ctypes.c_int * b)(*[int(x) for x in ns])
    PA = (ctypes.c_void_p * b)(*[_dev(a, "A")[0] for a in As])
    PQ = (ctypes.c_void_p * b)(*[_dev(q, "Q")[0] for q in Qs])
    PH = (ctypes.c_void_p * b)(*[_dev(q, "Qhat")[0] for q in Qhats]) if Qhats is not None else None
    it = (ctypes.c_int * b)()
    stv = (ctypes.c_int * b)()
    s = lib().schur_refine_batched(h, b, N, PA, PQ, PH, it, stv)
    return s, list(it), list(stv)


def schur_refine_residuals(h, n: int, A, Q):
    """Returns (status, stril_rel, orth)."""
    pa, lda = _dev(A, "A")
    pq, ldq = _dev(Q, "Q")
    a, b = ctypes.c_double(), ctypes.c_double()
    s = lib().schur_refine_residuals(h, int(n), pa, lda, pq, ldq, ctypes.byref(a), ctypes.byref(b))
    return s, a.value, b.value


def schur_refine_residuals_noalloc(n: int, A, Q, stream=None):
    """Residuals without a handle or any device allocation (n <= 512).

    For callers that cannot allocate device memory (their memory belongs to a
    pool allocator, or allocation is forbidden after start-up). Returns
    (status, stril_rel, orth).
    """
    pa, lda = _dev(A, "A")
    pq, ldq = _dev(Q, "Q")
    a, b = ctypes.c_double(), ctypes.c_double()
    st = ctypes.c_void_p(int(stream)) if stream is not None else None
    s = lib().schur_refine_residuals_noalloc(int(n), pa, lda, pq, ldq, ctypes.byref(a), ctypes.byref(b), st)
    return s, a.value, b.value


def schur_refine_trisolve(h, n: int, TE, diag):
    pt, ld = _dev(TE, "TE")
    pd, _ = _dev(diag, "diag")
    return lib().schur_refine_trisolve(h, int(n), pt, ld, pd)


def schur_refine_solve_plan(n: int):
    """The dataflow solve's task list for order n (numpy uint64 array)."""
    import numpy as np
    cnt = ctypes.c_longlong(0)
    s = lib().schur_refine_solve_plan(int(n), None, 0, ctypes.byref(cnt))
    if s != 0:
        raise SchurRefineError(s, "schur_refine_solve_plan")
    out = np.zeros(cnt.value, dtype=np.uint64)
    s = lib().schur_refine_solve_plan(int(n), out.ctypes.data_as(ctypes.POINTER(ctypes.c_ulonglong)), cnt.value,
                                      ctypes.byref(cnt))
    if s != 0:
        raise SchurRefineError(s, "schur_refine_solve_plan")
    return out


def schur_refine_crt_info(N: int, limbs: int, K: int):
    """(status, moduli, weights as Python ints, M as a Python int, sigma, t) of the
    residue form's table (host code; no device)."""
    mod = (ctypes.c_int * max(N, 1))()
    w = (ctypes.c_uint * max(N * limbs, 1))()
    M = (ctypes.c_uint * max(limbs, 1))()
    sg, t = ctypes.c_int(0), ctypes.c_int(0)
    s = lib().schur_refine_crt_info(int(N), int(limbs), int(K), mod, w, M, ctypes.byref(sg), ctypes.byref(t))
    if s != 0:
        return s, None, None, None, None, None

    def big(limbs_):
        return sum(int(x) << (32 * k) for k, x in enumerate(limbs_))

    weights = [big(w[l * limbs:(l + 1) * limbs]) for l in range(N)]
    return s, list(mod[:N]), weights, big(M[:limbs]), sg.value, t.value


def schur_refine_selftest_wait_timeout(h):
    return lib().schur_refine_selftest_wait_timeout(h)


def schur_refine_gemm(h, transA: int, m: int, n: int, k: int, A, B, C):
    pa, lda = _dev(A, "A")
    pb, ldb = _dev(B, "B")
    pc, ldc = _dev(C, "C")
    return lib().schur_refine_gemm(h, int(transA), int(m), int(n), int(k), pa, lda, pb, ldb, pc, ldc)


def schur_refine_get_profile(h):
    p = sr_profile()
    s = lib().schur_refine_get_profile(h, ctypes.byref(p))
    return s, p


def schur_refine_reset_profile(h):
    return lib().schur_refine_reset_profile(h)


def schur_refine_destroy(h):
    lib().schur_refine_destroy(h)
