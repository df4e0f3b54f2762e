"""CPU oracle for the Schur refinement iteration -- TEST INFRASTRUCTURE ONLY.

Plain numpy (matrix products as library primitives) plus the C routines of
``schur_oracle.c`` for the triangular solve and double-double residuals. Only
the tests, the smoke check and the benchmark's CPU-baseline leg may import
this module; the product path never does.

Every function follows the paper's steps in its order and notation:

* :func:`ns_init`      -- Alg. 4 line "convert Qhat to hp, one Newton-Schulz
  step", eq. (NS) of Sec. 2.4: Q = 1/2 Qhat (3I - Qhat^H Qhat).
* :func:`alg2`         -- Alg. 2 (successive substitution) for
  stril(T L - L T) = -E, eq. (2.5) of Sec. 2.1.
* :func:`alg3`         -- Alg. 3 (recursive block algorithm), Sec. 2.1.
* :func:`kron_solve`   -- brute force of the same equation (dense solve of the
  operator's n(n-1)/2-square matrix in 128-bit arithmetic).
* :func:`alg2_quasi`   -- Alg. 2 for the real quasi-triangular Schur form of
  Sec. 3 (2 x 2 diagonal blocks for complex-conjugate pairs; blocks read off
  T^ by :func:`quasi_blocks`).
* :func:`sym_solve`    -- Sec. 2.5 (symmetric A): with T diagonal the equation
  decouples, l_ij = -e_ij / (t_ii - t_jj) for i > j (the sign of eq. (lij)).
* :func:`iteration`    -- one pass of the REPEAT loop of Alg. 4 (Sec. 2.4):
  T^ = Q^H A Q in hp; E = stril(T^), T = T^ - E, to lp; solve in lp; L to
  hp; W = L - L^H; Y = Q^H Q - I in hp; YW, W^2, W^3 in lp; Sigma in hp;
  Q <- 1/2 Q Sigma in hp (eq. "NSmerged", truncated as Sec. 2.4 states).
* :func:`refine`       -- Alg. 4 from Qhat until the stop test holds.
* :func:`residuals_dd` -- ||stril(Q^H A Q)||_F / ||A||_F and ||Q^H Q - I||_F
  (the two error measures of Sec. 3) in double-double.

Precision pairs: hp is float64 (complex128); lp is float32 (complex64) for the
mixed form and float64 (complex128) for the all-FP64 form.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import _lib

OK, NONDISTINCT, NONFINITE, NOT_CONVERGED = 0, 2, 3, 4


class SolveError(RuntimeError):
    def __init__(self, code: int):
        super().__init__({NONDISTINCT: "diagonal entries of T are not pairwise distinct (Theorem 1)",
                          NONFINITE: "non-finite value in the solution"}.get(code, f"code {code}"))
        self.code = code


def _lp_dtype(lp: str, complex_: bool):
    if lp == "f32":
        return np.complex64 if complex_ else np.float32
    if lp == "f64":
        return np.complex128 if complex_ else np.float64
    raise ValueError(lp)


def _hp_dtype(complex_: bool):
    return np.complex128 if complex_ else np.float64


def _ctype(a: np.ndarray):
    return a.dtype


# ---------------------------------------------------------------------------
# Triangular matrix equation stril(T L - L T) = -E  (Sec. 2.1)

def alg2(T: np.ndarray, E: np.ndarray, d_hp: np.ndarray | None = None, cap: float = 0.0,
         ncols: int | None = None) -> np.ndarray:
    """Alg. 2 in the precision of ``T`` (float32/64, complex64/128).

    ``d_hp`` is the diagonal of T in high precision; when given, the divisors
    t_ii - t_jj are formed from it and then rounded to the precision of T.
    ``cap`` > 0 applies the trick of Example 4 (Sec. 3): an entry of L larger
    than ``cap`` in modulus (|l|^2 > cap^2 for complex data, in the working
    precision) is set to zero as soon as it is computed, before later entries
    use it. ``ncols`` limits the solve to the columns j < ncols of L (the
    others are returned as zero): Alg. 2 forms column j from the columns
    before it only, so these are the leading columns of the full solve.
    Raises :class:`SolveError` on a zero divisor (Theorem 1) or a
    non-finite L.
    """
    n = T.shape[0]
    dt = T.dtype
    T = _lib.fortran(T, dt)
    E = _lib.fortran(E, dt)
    L = np.zeros((n, n), dtype=dt, order="F")
    L_ = _lib.lib()
    if np.iscomplexobj(T):
        dh = None if d_hp is None else np.ascontiguousarray(d_hp, dtype=np.complex128)
        fn = L_.sro_alg2_c64 if dt == np.complex64 else L_.sro_alg2_c128
    else:
        dh = None if d_hp is None else np.ascontiguousarray(d_hp, dtype=np.float64)
        fn = L_.sro_alg2_f32 if dt == np.float32 else L_.sro_alg2_f64
    rc = fn(n, _lib.ptr(T), n, _lib.ptr(E), n, None if dh is None else _lib.ptr(dh),
            _lib.ptr(L), n, float(cap), -1 if ncols is None else int(ncols))
    if rc:
        raise SolveError(rc)
    return L


def alg3(T: np.ndarray, E: np.ndarray, nmin: int = 2) -> np.ndarray:
    """Alg. 3 (recursive blocks, n1 = floor(n/2)) in float64."""
    n = T.shape[0]
    T = _lib.fortran(T, np.float64)
    Ew = _lib.fortran(E, np.float64).copy(order="F")
    L = np.zeros((n, n), order="F")
    rc = _lib.lib().sro_alg3_f64(n, _lib.ptr(T), n, _lib.ptr(Ew), n, _lib.ptr(L), n, int(nmin))
    if rc:
        raise SolveError(rc)
    return L


def kron_solve(T: np.ndarray, E: np.ndarray):
    """Brute-force solve in 128-bit arithmetic; returns (hi, lo) float64 planes."""
    n = T.shape[0]
    T = _lib.fortran(T, np.float64)
    E = _lib.fortran(E, np.float64)
    hi = np.zeros((n, n), order="F")
    lo = np.zeros((n, n), order="F")
    rc = _lib.lib().sro_kron_solve(n, _lib.ptr(T), n, _lib.ptr(E), n, _lib.ptr(hi), _lib.ptr(lo), n)
    if rc:
        raise SolveError(rc)
    return hi, lo


# ---------------------------------------------------------------------------
# Alg. 4 (Sec. 2.4)

def ns_init(Qhat: np.ndarray):
    """Convert Qhat to hp and apply one Newton-Schulz step, eq. (NS).

    Returns (Q, ||Qhat^H Qhat - I||_F), the latter measured in hp.
    """
    cplx = np.iscomplexobj(Qhat)
    Q = np.asfortranarray(Qhat.astype(_hp_dtype(cplx)))
    n = Q.shape[0]
    I = np.eye(n, dtype=Q.dtype)
    G = Q.conj().T @ Q
    y = float(np.linalg.norm(G - I))
    return np.asfortranarray(0.5 * (Q @ (3.0 * I - G))), y


@dataclass
class IterInfo:
    r_T: float                 # ||stril(Q^H A Q)||_F / ||A||_F of the incoming Q (hp)
    y_norm: float = math.nan   # ||Q^H Q - I||_F of the incoming Q (hp), nan if not formed
    w_norm: float = math.nan   # ||W||_F
    updated: bool = False


def sym_solve(E: np.ndarray, d_hp: np.ndarray, cap: float = 0.0) -> np.ndarray:
    """Sec. 2.5: the solution of stril(T L - L T) = -E for diagonal T, in the
    precision of ``E``: l_ij = -e_ij / (t_ii - t_jj) for i > j, each divisor
    formed from the hp diagonal ``d_hp`` and rounded to that precision (as in
    :func:`alg2`). For Hermitian A (complex ``E``) the Schur form is real
    diagonal, so the divisor is formed from the real parts of ``d_hp`` and
    divides the real and imaginary parts of e_ij separately. Raises
    :class:`SolveError` like alg2."""
    n = E.shape[0]
    dt = E.dtype
    L = np.zeros((n, n), dtype=dt)
    i, j = np.tril_indices(n, -1)
    cplx = np.iscomplexobj(E)
    if cplx:
        rt = np.float32 if dt == np.complex64 else np.float64
        dr = np.real(np.asarray(d_hp)).astype(np.float64)
        den = (dr[i] - dr[j]).astype(rt)
    else:
        den = (np.asarray(d_hp)[i] - np.asarray(d_hp)[j]).astype(dt)
    if np.any(den == 0):
        raise SolveError(NONDISTINCT)
    with np.errstate(over="ignore", invalid="ignore"):
        if cplx:
            e = E[i, j]
            vals = np.empty(len(i), dtype=dt)
            vals.real = -(e.real / den)
            vals.imag = -(e.imag / den)
        else:
            vals = -E[i, j] / den
    if cap > 0:   # the trick of Example 4, as in alg2 (|l|^2 > cap^2 for complex data)
        if cplx:
            rt = vals.real.dtype.type
            vals[vals.real * vals.real + vals.imag * vals.imag > rt(cap) * rt(cap)] = 0
        else:
            vals[np.abs(vals) > dt.type(cap)] = 0
    if not np.all(np.isfinite(vals)):
        raise SolveError(NONFINITE)
    L[i, j] = vals
    return L


def quasi_blocks(That: np.ndarray) -> np.ndarray:
    """Diagonal block sizes of a real quasi-triangular Schur form read off T^
    (Sec. 3, real Schur decompositions): blk[k] = 2 when rows k, k+1 form a 2 x 2
    block, with blk[k + 1] = 0, else 1. Rows are taken from the top; rows k, k+1
    form a block when the 2 x 2 diagonal block of T^ there has non-real
    eigenvalues, (t_kk - t_k+1,k+1)^2 + 4 t_k,k+1 t_k+1,k < 0 (evaluated in hp)."""
    n = That.shape[0]
    blk = np.ones(n, dtype=np.int32)
    k = 0
    while k < n:
        if k + 1 < n:
            a, b, c, d = That[k, k], That[k, k + 1], That[k + 1, k], That[k + 1, k + 1]
            if (a - d) * (a - d) + 4.0 * b * c < 0.0:
                blk[k], blk[k + 1] = 2, 0
                k += 2
                continue
        k += 1
    return blk


def block_lower_mask(blk: np.ndarray) -> np.ndarray:
    """Mask of the entries below the diagonal blocks (the strictly block-lower part)."""
    n = len(blk)
    owner = np.arange(n)
    for k in range(n):
        if blk[k] == 0:
            owner[k] = k - 1
    return owner[:, None] > owner[None, :]


def form_residual(A: np.ndarray, Q: np.ndarray, quasi: bool = False):
    """T^ = Q^H A Q in hp (two products), split into E = stril(T^) and T = T^ - E.
    With ``quasi`` (real quasi-triangular Schur form), E is the strictly
    block-lower part for the blocks :func:`quasi_blocks` reads off T^, and the
    block sizes are returned third."""
    That = Q.conj().T @ (A @ Q)
    if quasi:
        blk = quasi_blocks(That)
        E = np.where(block_lower_mask(blk), That, 0.0)
        return That - E, E, blk
    E = np.tril(That, -1)
    T = That - E
    return T, E


def alg2_quasi(T: np.ndarray, E: np.ndarray, blk: np.ndarray, d_hp: np.ndarray, cap: float = 0.0) -> np.ndarray:
    """Alg. 2 for the real quasi-triangular form in the precision of ``T``
    (float32/64): sbl(T L - L T) = -E for strictly block-lower L, block columns
    left to right and block rows bottom to top, each block equation
    T_II X - X T_JJ = -C_IJ solved through its Kronecker matrix (at most 4 x 4)
    whose diagonal entries t_rr - t_cc are formed from the hp diagonal ``d_hp``
    and rounded once, by Gaussian elimination with partial pivoting. With every
    block 1 x 1 it is :func:`alg2`. Raises :class:`SolveError` on a shared
    eigenvalue of two blocks (a zero pivot) or a non-finite L."""
    n = T.shape[0]
    dt = T.dtype
    T = _lib.fortran(T, dt)
    E = _lib.fortran(E, dt)
    L = np.zeros((n, n), dtype=dt, order="F")
    dh = np.ascontiguousarray(d_hp, dtype=np.float64)
    b = np.ascontiguousarray(blk, dtype=np.int32)
    fn = _lib.lib().sro_alg2_quasi_f32 if dt == np.float32 else _lib.lib().sro_alg2_quasi_f64
    rc = fn(n, _lib.ptr(T), n, _lib.ptr(E), n, _lib.ptr(dh), _lib.ptr(b), _lib.ptr(L), n, float(cap))
    if rc:
        raise SolveError(rc)
    return L


def iteration(A: np.ndarray, Q: np.ndarray, lp: str = "f32", full_sigma: bool = False,
              solver: str = "alg2", T_E=None, parts: dict | None = None, symmetric: bool = False,
              cap: float = 0.0, quasi: bool = False):
    """One pass of the REPEAT loop of Alg. 4; returns (Q_new, IterInfo).

    ``full_sigma`` adds the two terms W^2 Y + W^2 Y W that Sec. 2.4 drops.
    ``symmetric`` takes Sec. 2.5's form for real symmetric A: T is the
    diagonal of T^ and the solve is :func:`sym_solve`. ``cap`` is the entry
    threshold of :func:`alg2`.
    If ``parts`` is a dict, the intermediates T, E, L, W, Y and Sigma are
    stored in it.
    """
    cplx = np.iscomplexobj(A)
    hp = _hp_dtype(cplx)
    lpt = _lp_dtype(lp, cplx)
    n = A.shape[0]
    I = np.eye(n, dtype=hp)
    if quasi:
        T, E, blk = form_residual(A, Q, quasi=True) if T_E is None else T_E
    else:
        T, E = form_residual(A, Q) if T_E is None else T_E
    info = IterInfo(r_T=float(np.linalg.norm(E) / np.linalg.norm(A)))
    # E, T to lp; divisors from the hp diagonal
    T_lp = np.asfortranarray(T.astype(lpt))
    E_lp = np.asfortranarray(E.astype(lpt))
    if symmetric:
        L_lp = sym_solve(E_lp, np.diagonal(T).copy(), cap)
    elif quasi:
        L_lp = alg2_quasi(T_lp, E_lp, blk, np.diagonal(T).copy(), cap)
    elif solver == "alg2":
        L_lp = alg2(T_lp, E_lp, np.diagonal(T).copy(), cap)
    elif solver == "alg3":
        if lpt != np.float64:
            raise ValueError("alg3 oracle is float64 only")
        L_lp = alg3(T_lp, E_lp)
    else:
        raise ValueError(solver)
    L = L_lp.astype(hp)
    W = L - L.conj().T
    Y = Q.conj().T @ Q - I
    info.y_norm = float(np.linalg.norm(Y))
    info.w_norm = float(np.linalg.norm(W))
    # products in lp
    Y_l = Y.astype(lpt)
    W_l = W.astype(lpt)
    YW = Y_l @ W_l
    W2 = W_l @ W_l
    W3 = W_l @ W2
    Sigma = 2.0 * I + 2.0 * W - Y - YW.astype(hp) + W2.astype(hp) + W3.astype(hp)
    if full_sigma:
        W2Y = W2 @ Y_l
        W2YW = W2Y @ W_l
        Sigma = Sigma + W2Y.astype(hp) + W2YW.astype(hp)
    Qn = np.asfortranarray(0.5 * (Q @ Sigma))
    info.updated = True
    if parts is not None:
        parts.update(T=T, E=E, L=L, W=W, Y=Y, Sigma=Sigma)
    return Qn, info


def default_tol(n: int) -> float:
    """FP64 target: 1e-14 sqrt(n)."""
    return 1e-14 * math.sqrt(n)


@dataclass
class RefineResult:
    Q: np.ndarray
    status: int
    iters: int                     # number of T^ formations
    hp_gemms: int                  # high-precision matrix products
    history: list = field(default_factory=list)
    y0: float = math.nan


def refine(A: np.ndarray, Qhat: np.ndarray, lp: str = "f32", tol: float | None = None,
           max_iter: int = 10, full_sigma: bool = False, solver: str = "alg2",
           init_ns: bool = True, symmetric: bool = False, cap: float = 0.0,
           quasi: bool = False) -> RefineResult:
    """Alg. 4 lines "convert Qhat, NS step" and REPEAT ... UNTIL convergence.

    Stop test (the paper only says "when E becomes small enough"): after
    forming T^ from Q_k, stop if ||E||_F / ||A||_F <= tol and the last
    measured ||Q^H Q - I||_F <= sqrt(tol). The final pass forms T^ only, so a
    run of k passes costs 2 + 4(k-1) + 2 = 4k high-precision products when it
    starts with the Newton-Schulz step.
    """
    n = A.shape[0]
    tol = default_tol(n) if tol is None else tol
    if init_ns:
        Q, y = ns_init(Qhat)
        gemms = 2
    else:
        Q = np.asfortranarray(Qhat.astype(_hp_dtype(np.iscomplexobj(A))))
        y, gemms = math.nan, 0
    res = RefineResult(Q=Q, status=NOT_CONVERGED, iters=0, hp_gemms=gemms, y0=y)
    y_last = y
    prev_rT = math.inf
    for k in range(1, max_iter + 1):
        TE = form_residual(A, Q, quasi=quasi)
        T, E = TE[0], TE[1]
        res.hp_gemms += 2
        res.iters = k
        r_T = float(np.linalg.norm(E) / np.linalg.norm(A))
        if not math.isfinite(r_T):
            res.status = NONFINITE
            res.history.append(IterInfo(r_T=r_T))
            break
        ok_y = (not math.isfinite(y_last)) or y_last <= math.sqrt(tol)
        if r_T <= tol and ok_y:
            res.status = OK
            res.history.append(IterInfo(r_T=r_T))
            break
        if k >= 3 and r_T > 10.0 * prev_rT:
            res.status = NOT_CONVERGED
            res.history.append(IterInfo(r_T=r_T))
            break
        prev_rT = r_T
        try:
            Q, info = iteration(A, Q, lp=lp, full_sigma=full_sigma, solver=solver, T_E=TE,
                                symmetric=symmetric, cap=cap, quasi=quasi)
        except SolveError as e:
            res.status = e.code
            res.history.append(IterInfo(r_T=r_T))
            break
        res.hp_gemms += 2
        res.history.append(info)
        y_last = info.y_norm
        res.Q = Q
        if not np.all(np.isfinite(Q)):
            res.status = NONFINITE
            break
    return res


# ---------------------------------------------------------------------------
# Residuals in double-double (Sec. 3 error measures)

def residuals_dd(A: np.ndarray, Q: np.ndarray, threads: int | None = None, blk: np.ndarray | None = None):
    """(r_T, r_Q) = (||stril(Q^H A Q)||_F/||A||_F, ||Q^H Q - I||_F) in double-double.
    With ``blk`` (real quasi-triangular form, see :func:`quasi_blocks`) r_T is
    the norm of the entries below the diagonal blocks."""
    n = A.shape[0]
    if threads is not None:
        _lib.set_threads(threads)
    rT = np.zeros(1)
    rQ = np.zeros(1)
    if blk is not None:
        Af = _lib.fortran(A, np.float64)
        Qf = _lib.fortran(Q, np.float64)
        b = np.ascontiguousarray(blk, dtype=np.int32)
        _lib.lib().sro_residuals_dd_quasi(n, _lib.ptr(Af), n, _lib.ptr(Qf), n, _lib.ptr(b), _lib.ptr(rT),
                                          _lib.ptr(rQ))
        return float(rT[0]), float(rQ[0])
    if np.iscomplexobj(A) or np.iscomplexobj(Q):
        Af = _lib.fortran(A, np.complex128)
        Qf = _lib.fortran(Q, np.complex128)
        _lib.lib().sro_residuals_dd_c(n, _lib.ptr(Af), n, _lib.ptr(Qf), n, _lib.ptr(rT), _lib.ptr(rQ))
    else:
        Af = _lib.fortran(A, np.float64)
        Qf = _lib.fortran(Q, np.float64)
        _lib.lib().sro_residuals_dd(n, _lib.ptr(Af), n, _lib.ptr(Qf), n, _lib.ptr(rT), _lib.ptr(rQ))
    return float(rT[0]), float(rQ[0])


def sample_entries_dd(A: np.ndarray, Q: np.ndarray, rows, cols):
    """Entries (Q^H A Q)[rows, cols] and (Q^H Q - I)[rows, cols] in double-double
    (complex128 results for complex input)."""
    n = A.shape[0]
    r = np.ascontiguousarray(rows, dtype=np.int32)
    c = np.ascontiguousarray(cols, dtype=np.int32)
    if np.iscomplexobj(A) or np.iscomplexobj(Q):
        Af = _lib.fortran(A, np.complex128)
        Qf = _lib.fortran(Q, np.complex128)
        t = np.zeros(len(r), dtype=np.complex128)
        y = np.zeros(len(r), dtype=np.complex128)
        _lib.lib().sro_sample_entries_dd_c(n, _lib.ptr(Af), n, _lib.ptr(Qf), n, len(r), _lib.ptr(r),
                                           _lib.ptr(c), _lib.ptr(t), _lib.ptr(y))
        return t, y
    Af = _lib.fortran(A, np.float64)
    Qf = _lib.fortran(Q, np.float64)
    t = np.zeros(len(r))
    y = np.zeros(len(r))
    _lib.lib().sro_sample_entries_dd(n, _lib.ptr(Af), n, _lib.ptr(Qf), n, len(r), _lib.ptr(r),
                                     _lib.ptr(c), _lib.ptr(t), _lib.ptr(y))
    return t, y


def gemm_dd(A_hi, A_lo, B_hi, B_lo, transA: bool = False):
    """C = op(A) B with double-double operands (lo planes may be None)."""
    m = A_hi.shape[1] if transA else A_hi.shape[0]
    k = A_hi.shape[0] if transA else A_hi.shape[1]
    n = B_hi.shape[1]
    Ah = _lib.fortran(A_hi, np.float64)
    Al = None if A_lo is None else _lib.fortran(A_lo, np.float64)
    Bh = _lib.fortran(B_hi, np.float64)
    Bl = None if B_lo is None else _lib.fortran(B_lo, np.float64)
    Ch = np.zeros((m, n), order="F")
    Cl = np.zeros((m, n), order="F")
    _lib.lib().sro_gemm_dd(int(transA), m, n, k, _lib.ptr(Ah), None if Al is None else _lib.ptr(Al),
                           Ah.shape[0], _lib.ptr(Bh), None if Bl is None else _lib.ptr(Bl),
                           Bh.shape[0], _lib.ptr(Ch), _lib.ptr(Cl), m)
    return Ch, Cl
