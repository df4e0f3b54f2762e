"""Alg. 4 with double-double working precision -- TEST INFRASTRUCTURE ONLY.

The high precision (hp) is double-double: a pair of float64 arrays (hi, lo)
stands for hi + lo. The low precision (lp) is float64. Every hp product is the
plain triple loop of ``sro_gemm_dd`` (TwoProd/TwoSum, Dekker and Knuth), the
solve is Alg. 2 in float64 (``sro_alg2_f64_dd``), and the error measures of
Sec. 3 are evaluated in 128-bit floating point (``sro_residuals_q``,
``sro_sample_entries_q``). Elementwise double-double sums are written out
below. Only the tests and the benchmark's CPU-baseline leg use this module.

Steps, in the order of Alg. 4 (Sec. 2.4):
  * :func:`ns_init_dd`    -- Qhat to hp, Q = 1/2 Qhat (3I - Qhat^T Qhat) (eq. NS).
  * :func:`iteration_dd`  -- T^ = Q^T (A Q) in hp; E = stril(T^), T = T^ - E,
    rounded to lp; Alg. 2 in lp; W = L - L^T; Y = Q^T Q - I in hp; YW, W^2,
    W^3 in lp; Sigma = 2I + 2W - Y - YW + W^2 + W^3 in hp; Q <- 1/2 Q Sigma in hp.
  * :func:`refine_dd`     -- the REPEAT loop with the stop test of the FP64
    forms and the tolerance 1e-28 n.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import _lib
from .alg import NONFINITE, NOT_CONVERGED, OK, IterInfo, SolveError


# ---- elementwise double-double arithmetic (Knuth TwoSum) ---------------------

def _two_sum(a, b):
    s = a + b
    bb = s - a
    return s, (a - (s - bb)) + (b - bb)


def _renorm(a, b):
    s = a + b
    return s, b - (s - a)


def dd_add(x, y):
    """(xh + xl) + (yh + yl) in double-double; x, y are (hi, lo) pairs."""
    s, e = _two_sum(x[0], y[0])
    t, f = _two_sum(x[1], y[1])
    s, e = _renorm(s, e + t)
    return _renorm(s, e + f)


def dd_neg(x):
    return (-x[0], -x[1])


def dd_scale(x, c):
    """c * x for a power of two c (exact)."""
    return (c * x[0], c * x[1])


def dd_value_norm(x) -> float:
    """Frobenius norm of hi + lo (the sum rounded to float64 first)."""
    return float(np.linalg.norm(x[0] + x[1]))


def dd(x):
    return (np.asfortranarray(x, dtype=np.float64), np.zeros_like(x, dtype=np.float64, order="F"))


def gemm(x, y, transA: bool = False):
    """op(X) Y in double-double with the oracle's triple loop."""
    xh = _lib.fortran(x[0], np.float64)
    xl = _lib.fortran(x[1], np.float64)
    yh = _lib.fortran(y[0], np.float64)
    yl = _lib.fortran(y[1], np.float64)
    m = xh.shape[1] if transA else xh.shape[0]
    k = xh.shape[0] if transA else xh.shape[1]
    n = yh.shape[1]
    ch = np.zeros((m, n), order="F")
    cl = np.zeros((m, n), order="F")
    _lib.lib().sro_gemm_dd(int(transA), m, n, k, _lib.ptr(xh), _lib.ptr(xl), xh.shape[0], _lib.ptr(yh),
                           _lib.ptr(yl), yh.shape[0], _lib.ptr(ch), _lib.ptr(cl), m)
    return ch, cl


def alg2_dd_divisors(T: np.ndarray, E: np.ndarray, d, cap: float = 0.0) -> np.ndarray:
    """Alg. 2 in float64 with divisors t_ii - t_jj from the double-double diagonal d."""
    n = T.shape[0]
    T = _lib.fortran(T, np.float64)
    E = _lib.fortran(E, np.float64)
    dh = np.ascontiguousarray(d[0], dtype=np.float64)
    dl = np.ascontiguousarray(d[1], dtype=np.float64)
    L = np.zeros((n, n), order="F")
    rc = _lib.lib().sro_alg2_f64_dd(n, _lib.ptr(T), n, _lib.ptr(E), n, _lib.ptr(dh), _lib.ptr(dl),
                                    _lib.ptr(L), n, float(cap))
    if rc:
        raise SolveError(rc)
    return L


def residuals_q(A, Q):
    """(r_T, r_Q) of Sec. 3 for double-double A and Q, in 128-bit arithmetic."""
    n = A[0].shape[0]
    f = lambda x: _lib.fortran(x, np.float64)
    Ah, Al, Qh, Ql = f(A[0]), f(A[1]), f(Q[0]), f(Q[1])
    rT = np.zeros(1)
    rQ = np.zeros(1)
    _lib.lib().sro_residuals_q(n, _lib.ptr(Ah), _lib.ptr(Al), n, _lib.ptr(Qh), _lib.ptr(Ql), n,
                               _lib.ptr(rT), _lib.ptr(rQ))
    return float(rT[0]), float(rQ[0])


def sample_entries_q(A, Q, rows, cols):
    """Entries (Q^T A Q)[rows, cols] and (Q^T Q - I)[rows, cols] in 128-bit
    arithmetic, each returned as a double-double pair of arrays."""
    n = A[0].shape[0]
    f = lambda x: _lib.fortran(x, np.float64)
    Ah, Al, Qh, Ql = f(A[0]), f(A[1]), f(Q[0]), f(Q[1])
    r = np.ascontiguousarray(rows, dtype=np.int32)
    c = np.ascontiguousarray(cols, dtype=np.int32)
    out = [np.zeros(len(r)) for _ in range(4)]
    _lib.lib().sro_sample_entries_q(n, _lib.ptr(Ah), _lib.ptr(Al), n, _lib.ptr(Qh), _lib.ptr(Ql), n, len(r),
                                    _lib.ptr(r), _lib.ptr(c), *[_lib.ptr(o) for o in out])
    return (out[0], out[1]), (out[2], out[3])


def _eye_dd(n):
    return dd(np.eye(n))


# ---- Alg. 4 --------------------------------------------------------------------

def ns_init_dd(Qhat: np.ndarray):
    """eq. (NS) in double-double: Q = 1/2 Qhat (3I - Qhat^T Qhat).

    Returns (Q, ||Qhat^T Qhat - I||_F)."""
    n = Qhat.shape[0]
    Q = dd(Qhat)
    G = gemm(Q, Q, transA=True)
    Y = dd_add(G, dd_neg(_eye_dd(n)))
    M = dd_add(dd_scale(_eye_dd(n), 3.0), dd_neg(G))
    return dd_scale(gemm(Q, M), 0.5), dd_value_norm(Y)


def form_residual_dd(A, Q):
    """T^ = Q^T (A Q) in double-double, split into E = stril(T^) and T = T^ - E."""
    That = gemm(Q, gemm(A, Q), transA=True)
    E = (np.tril(That[0], -1), np.tril(That[1], -1))
    T = (np.triu(That[0]), np.triu(That[1]))
    return T, E


def _round(x):
    """Double-double to float64: hi + lo rounded."""
    return np.asfortranarray(x[0] + x[1])


def iteration_dd(A, Q, full_sigma: bool = False, T_E=None, parts: dict | None = None):
    """One pass of the REPEAT loop of Alg. 4 with hp = double-double, lp = float64."""
    n = A[0].shape[0]
    I = np.eye(n)
    T, E = form_residual_dd(A, Q) if T_E is None else T_E
    info = IterInfo(r_T=dd_value_norm(E) / dd_value_norm(A))
    T_lp, E_lp = _round(T), _round(E)
    d = (np.diagonal(T[0]).copy(), np.diagonal(T[1]).copy())
    L = alg2_dd_divisors(T_lp, E_lp, d)
    W = L - L.T
    Y = dd_add(gemm(Q, Q, transA=True), dd_neg(_eye_dd(n)))
    info.y_norm = dd_value_norm(Y)
    info.w_norm = float(np.linalg.norm(W))
    # products in lp
    Y_l = _round(Y)
    YW = Y_l @ W
    W2 = W @ W
    W3 = W @ W2
    S = dd(2.0 * I)
    S = dd_add(S, dd(2.0 * W))
    S = dd_add(S, dd_neg(Y))
    S = dd_add(S, dd(-YW))
    S = dd_add(S, dd(W2))
    S = dd_add(S, dd(W3))
    if full_sigma:
        W2Y = W2 @ Y_l
        S = dd_add(S, dd(W2Y))
        S = dd_add(S, dd(W2Y @ W))
    Qn = dd_scale(gemm(Q, S), 0.5)
    info.updated = True
    if parts is not None:
        parts.update(T=T, E=E, L=L, W=W, Y=Y, Sigma=S)
    return Qn, info


def default_tol_dd(n: int) -> float:
    """Double-double target: 1e-28 n."""
    return 1e-28 * n


@dataclass
class RefineResultDD:
    Q: tuple                       # (hi, lo)
    status: int
    iters: int
    hp_gemms: int
    history: list = field(default_factory=list)
    y0: float = math.nan


def refine_dd(A, Qhat: np.ndarray, tol: float | None = None, max_iter: int = 10,
              full_sigma: bool = False) -> RefineResultDD:
    """Alg. 4 from a float64 Qhat with hp = double-double and lp = float64.

    The stop test is that of the FP64 forms: after forming T^ from Q_k, stop
    if ||E||_F / ||A||_F <= tol and the last ||Q^T Q - I||_F <= sqrt(tol)."""
    n = A[0].shape[0]
    tol = default_tol_dd(n) if tol is None else tol
    Q, y = ns_init_dd(Qhat)
    res = RefineResultDD(Q=Q, status=NOT_CONVERGED, iters=0, hp_gemms=2, y0=y)
    y_last = y
    prev = math.inf
    anorm = dd_value_norm(A)
    for k in range(1, max_iter + 1):
        T, E = form_residual_dd(A, Q)
        res.hp_gemms += 2
        res.iters = k
        r_T = dd_value_norm(E) / anorm
        if not math.isfinite(r_T):
            res.status = NONFINITE
            res.history.append(IterInfo(r_T=r_T))
            break
        if r_T <= tol and y_last <= math.sqrt(tol):
            res.status = OK
            res.history.append(IterInfo(r_T=r_T))
            break
        if k >= 3 and r_T > 10.0 * prev:
            res.history.append(IterInfo(r_T=r_T))
            break
        prev = r_T
        try:
            Q, info = iteration_dd(A, Q, full_sigma=full_sigma, T_E=(T, E))
        except SolveError as e:
            res.status = e.code
            res.history.append(IterInfo(r_T=r_T))
            break
        res.hp_gemms += 2
        res.history.append(info)
        y_last = info.y_norm
        res.Q = Q
    return res
