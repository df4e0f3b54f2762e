"""Alg. 4 with a multi-word working precision -- TEST INFRASTRUCTURE ONLY.

Sec. 3 refines to working precisions held as several doubles per number (two
for quadruple precision, six for 100 digits). This module checks the
library's triple-double form (about 159 bits, F = 256) and six-double form
(about 318 bits, F = 512). It models the high precision
(hp) by exact binary fixed point: an hp matrix is a numpy object array of
Python integers X standing for X 2^-F, F = 256 fraction bits by default. Every
hp product is the exact integer matrix product, rounded once to the grid;
sums are exact. For entries of order one this is about 2^97 times finer than
a triple-double, so the oracle's hp is at least as accurate as the form it
checks and its result differs from the library's only by the library's own
rounding.

The low precision (lp) is float64, as in the library's multi-word forms:
  * T^ and E rounded to float64 (the nearest double to each entry),
  * Alg. 2 in float64 with each divisor t_ii - t_jj formed from the two
    leading words of the hp diagonal (``ddtarget.alg2_dd_divisors``),
  * W = L - L^T, and YW, W^2, W^3 as float64 products (numpy), with Y rounded
    to float64.

Steps, in the order of Alg. 4 (Sec. 2.4):
  * :func:`ns_init_fx`   -- Q = 1/2 Qhat (3I - Qhat^T Qhat) in hp (eq. NS).
  * :func:`iteration_fx` -- T^ = Q^T (A Q) in hp; E = stril(T^), T = T^ - E in
    lp; Alg. 2 in lp; W; Y = Q^T Q - I in hp; YW, W^2, W^3 in lp;
    Sigma = 2I + 2W - Y - YW + W^2 + W^3 in hp; Q <- 1/2 Q Sigma in hp.
  * :func:`refine_fx`    -- the REPEAT loop with the stop test of the other
    forms and the tolerance 1e-45 n.
  * :func:`residuals_exact` -- ||stril(Q^T A Q)||_F / ||A||_F and
    ||Q^T Q - I||_F of given A, Q evaluated exactly.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from fractions import Fraction

import numpy as np

from .alg import NONFINITE, NOT_CONVERGED, OK, IterInfo, SolveError
from .ddtarget import alg2_dd_divisors

FBITS = 256


# ---- exact conversions ---------------------------------------------------------

def _f2i(d: float, F: int) -> int:
    """The float d times 2^F rounded to the nearest integer (ties to even);
    exact whenever d has no bits below 2^-F."""
    if d == 0.0:
        return 0
    if not math.isfinite(d):
        raise ValueError("non-finite entry")
    m, e = math.frexp(d)               # d = m 2^e, 0.5 <= |m| < 1
    mant = int(m * (1 << 53))          # exact: m carries 53 bits
    sh = e - 53 + F
    if sh >= 0:
        return mant << sh
    return int(round(Fraction(mant, 1 << (-sh))))


_f2i_vec = np.frompyfunc(_f2i, 2, 1)


def to_fx(x, F: int = FBITS) -> np.ndarray:
    """Exact fixed-point image of a float64 array, or of a tuple of float64
    planes standing for their sum (a multi-word matrix)."""
    if isinstance(x, (tuple, list)):
        out = to_fx(x[0], F)
        for p in x[1:]:
            out = out + to_fx(p, F)
        return out
    a = np.asarray(x, dtype=np.float64)
    return _f2i_vec(a, F).astype(object)


def _nearest(X: int, F: int) -> float:
    """The double nearest to X 2^-F (Python's int / int division rounds once)."""
    return X / (1 << F) if F >= 0 else float(X << (-F))


_nearest_vec = np.frompyfunc(_nearest, 2, 1)


def to_float(X: np.ndarray, F: int = FBITS) -> np.ndarray:
    """Each entry X 2^-F rounded to the nearest double."""
    return np.asarray(_nearest_vec(X, F), dtype=np.float64)


def _words(X: int, F: int, k: int):
    r = Fraction(X, 1 << F)
    out = []
    for _ in range(k):
        w = float(r)                   # nearest double to what is left
        out.append(w)
        r -= Fraction(w)
    return out


def to_words(X: np.ndarray, F: int = FBITS, k: int = 3):
    """The k-word expansion of each entry: word 1 the double nearest to the
    value, each next word the double nearest to what the words before leave."""
    X = np.asarray(X, dtype=object)
    planes = [np.zeros(X.shape) for _ in range(k)]
    for idx in np.ndindex(X.shape):
        for p, w in zip(planes, _words(int(X[idx]), F, k)):
            p[idx] = w
    return tuple(np.asfortranarray(p) for p in planes)


def eye_fx(n: int, F: int = FBITS) -> np.ndarray:
    I = np.zeros((n, n), dtype=object)
    I[:] = 0
    for i in range(n):
        I[i, i] = 1 << F
    return I


def _round_shift(X: np.ndarray, s: int) -> np.ndarray:
    """X 2^-s rounded to the nearest integer (halves up)."""
    h = 1 << (s - 1)
    f = np.frompyfunc(lambda v: (v + h) >> s, 1, 1)
    return f(X).astype(object)


def matmul_fx(A: np.ndarray, B: np.ndarray, F: int = FBITS, extra: int = 0) -> np.ndarray:
    """The exact product (A 2^-F)(B 2^-F) times 2^-extra, rounded once to the
    grid 2^-F."""
    return _round_shift(np.dot(A, B), F + extra)


def norm_fx(X: np.ndarray, F: int = FBITS) -> float:
    """||X 2^-F||_F (the exact sum of squares, rounded once, then sqrt)."""
    s = sum(int(v) * int(v) for v in np.asarray(X, dtype=object).ravel())
    return math.sqrt(s / (1 << (2 * F))) if s else 0.0


# ---- Alg. 4 --------------------------------------------------------------------

def ns_init_fx(Qhat: np.ndarray, F: int = FBITS):
    """eq. (NS) in hp: Q = 1/2 Qhat (3I - Qhat^T Qhat). Returns (Q, ||Qhat^T Qhat - I||_F)."""
    n = Qhat.shape[0]
    Q = to_fx(Qhat, F)
    G = matmul_fx(Q.T, Q, F)
    I = eye_fx(n, F)
    Y = G - I
    return matmul_fx(Q, 3 * I - G, F, extra=1), norm_fx(Y, F)


def form_residual_fx(A: np.ndarray, Q: np.ndarray, F: int = FBITS):
    """T^ = Q^T (A Q) in hp, split into E = stril(T^) and T = T^ - E."""
    That = matmul_fx(Q.T, matmul_fx(A, Q, F), F)
    low = np.tril(np.ones(That.shape, dtype=bool), -1)
    E = np.where(low, That, 0).astype(object)
    T = np.where(low, 0, That).astype(object)
    return T, E


def iteration_fx(A: np.ndarray, Q: np.ndarray, F: int = FBITS, full_sigma: bool = False, T_E=None,
                 parts: dict | None = None):
    """One pass of the REPEAT loop of Alg. 4 with the fixed-point hp and lp = float64."""
    n = A.shape[0]
    T, E = form_residual_fx(A, Q, F) if T_E is None else T_E
    info = IterInfo(r_T=norm_fx(E, F) / norm_fx(A, F))
    T_lp, E_lp = to_float(T, F), to_float(E, F)
    dg = np.array([T[i, i] for i in range(n)], dtype=object)
    d0, d1 = to_words(dg, F, 2)
    L = alg2_dd_divisors(T_lp, E_lp, (d0, d1))
    W = L - L.T
    I = eye_fx(n, F)
    Y = matmul_fx(Q.T, Q, F) - I
    info.y_norm = norm_fx(Y, F)
    info.w_norm = float(np.linalg.norm(W))
    Y_l = to_float(Y, F)
    YW = Y_l @ W
    W2 = W @ W
    W3 = W @ W2
    S = 2 * I + to_fx(2.0 * W, F) - Y - to_fx(YW, F) + to_fx(W2, F) + to_fx(W3, F)
    if full_sigma:
        W2Y = W2 @ Y_l
        S = S + to_fx(W2Y, F) + to_fx(W2Y @ W, F)
    Qn = matmul_fx(Q, S, F, extra=1)
    info.updated = True
    if parts is not None:
        parts.update(T=T, E=E, L=L, W=W, Y=Y, Sigma=S)
    return Qn, info


def default_tol_td(n: int) -> float:
    """The triple-double target: 1e-45 n (about 700 n units of 2^-159). The
    passes from a float64 start reach about 1e-14, 1e-28, 1e-42 and then the
    working precision's floor: the tolerance lies inside the last gap, so the
    count of passes does not hang on the third pass's rounding."""
    return 1e-45 * n


def default_tol_d6(n: int) -> float:
    """The six-double target: 1e-93 n (about 500 n units of 2^-318). From a float64
    start the passes reach about 1e-14, 1e-28, ..., 1e-84 and then the working
    precision's floor near 1e-95: seven passes."""
    return 1e-93 * n


FBITS_D6 = 512   # fixed-point fraction bits for the six-double checks


@dataclass
class RefineResultFx:
    Q: np.ndarray                  # fixed point, 2^-F
    That: np.ndarray               # T^ of the last pass
    status: int
    iters: int
    hp_gemms: int
    F: int = FBITS
    history: list = field(default_factory=list)
    y0: float = math.nan


def refine_fx(A, Qhat: np.ndarray, tol: float | None = None, max_iter: int = 10, F: int = FBITS,
              full_sigma: bool = False) -> RefineResultFx:
    """Alg. 4 from a float64 Qhat with the fixed-point hp and lp = float64. A is a
    float64 array, a tuple of planes (a multi-word matrix) or a fixed-point array.

    The stop test is that of the other forms: after forming T^ from Q_k, stop
    if ||E||_F / ||A||_F <= tol and the last ||Q^T Q - I||_F <= sqrt(tol)."""
    A = A if (isinstance(A, np.ndarray) and A.dtype == object) else to_fx(A, F)
    n = A.shape[0]
    tol = default_tol_td(n) if tol is None else tol
    Q, y = ns_init_fx(Qhat, F)
    res = RefineResultFx(Q=Q, That=None, status=NOT_CONVERGED, iters=0, hp_gemms=2, F=F, y0=y)
    y_last = y
    prev = math.inf
    anorm = norm_fx(A, F)
    for k in range(1, max_iter + 1):
        T, E = form_residual_fx(A, Q, F)
        res.That = T + E
        res.hp_gemms += 2
        res.iters = k
        r_T = norm_fx(E, F) / anorm
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
            Q, info = iteration_fx(A, Q, F, full_sigma=full_sigma, T_E=(T, E))
        except SolveError as e:
            res.status = e.code
            res.history.append(IterInfo(r_T=r_T))
            break
        res.hp_gemms += 2
        res.history.append(info)
        y_last = info.y_norm
        res.Q = Q
    return res


def residuals_exact(A, Q, F: int = FBITS):
    """(r_T, r_Q) of Sec. 3 for A and Q (float64 arrays, tuples of planes or
    fixed-point arrays), each entry of Q^T A Q and Q^T Q - I formed exactly:
    r_T = ||stril(Q^T A Q)||_F / ||A||_F, r_Q = ||Q^T Q - I||_F."""
    A = A if (isinstance(A, np.ndarray) and A.dtype == object) else to_fx(A, F)
    Q = Q if (isinstance(Q, np.ndarray) and Q.dtype == object) else to_fx(Q, F)
    n = A.shape[0]
    M = np.dot(Q.T, np.dot(A, Q))                      # scale 2^-3F, exact
    low = np.tril(np.ones((n, n), dtype=bool), -1)
    sE = sum(int(v) * int(v) for v in M[low])
    rT = math.sqrt(sE / (1 << (6 * F))) / norm_fx(A, F) if sE else 0.0
    G = np.dot(Q.T, Q) - eye_fx(n, 2 * F)              # scale 2^-2F, exact
    sY = sum(int(v) * int(v) for v in G.ravel())
    rQ = math.sqrt(sY / (1 << (4 * F))) if sY else 0.0
    return rT, rQ
