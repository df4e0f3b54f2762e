"""Pins of the oracle for the real quasi-triangular Schur form (Sec. 3: real
Schur decompositions, whose 2 x 2 diagonal blocks hold complex-conjugate
pairs): the block solve sbl(T L - L T) = -E for strictly block-lower L
(sbl: the entries below the diagonal blocks) against a brute-force dense
solve in exact rational arithmetic, against Alg. 2 when every block is 1 x 1,
against a closed form and the equation itself, the failure when two blocks
share an eigenvalue, and the refinement against a planted decomposition."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2203_10879_gb300 import inputs


def _blocks_to_owner(blk):
    n = len(blk)
    return [k - 1 if blk[k] == 0 else k for k in range(n)]


def _quasi_problem(n, blk, seed, dt=np.float64):
    """Block upper triangular T with the given blocks (2 x 2 blocks with
    complex eigenvalues), E strictly block-lower."""
    rng = np.random.default_rng(seed)
    mu = np.sort(rng.uniform(0.0, 2.0, n)) + np.arange(n) * 0.3
    T = np.triu(rng.standard_normal((n, n)) * 0.3, 1)
    for k in range(n):
        if blk[k] == 2:
            a = 0.5 * (mu[k] + mu[k + 1])
            b = 0.2 + 0.3 * rng.uniform()
            T[k, k] = T[k + 1, k + 1] = a
            T[k, k + 1], T[k + 1, k] = b * 1.5, -b / 1.5
        elif blk[k] == 1:
            T[k, k] = mu[k]
    mask = oracle.block_lower_mask(np.asarray(blk))
    E = np.where(mask, rng.standard_normal((n, n)), 0.0)
    return T.astype(dt), E.astype(dt), np.diagonal(T).astype(np.float64).copy()


def _exact_block_solve(T, E, blk):
    """Brute force: the operator L -> sbl(T L - L T) on the strictly block-lower
    unknowns, assembled and solved in exact rational arithmetic."""
    n = T.shape[0]
    own = _blocks_to_owner(blk)
    unk = [(i, j) for j in range(n) for i in range(n) if own[i] > own[j]]
    N = len(unk)
    Tf = [[Fraction(float(T[i, j])) for j in range(n)] for i in range(n)]
    M = [[Fraction(0)] * (N + 1) for _ in range(N)]
    for c, (ui, uj) in enumerate(unk):
        # (T U - U T)(i, j) with U = e_ui e_uj^T: T[i, ui] [j == uj] - [i == ui] T[uj, j]
        for r, (i, j) in enumerate(unk):
            v = Fraction(0)
            if j == uj:
                v += Tf[i][ui]
            if i == ui:
                v -= Tf[uj][j]
            M[r][c] = v
    for r, (i, j) in enumerate(unk):
        M[r][N] = -Fraction(float(E[i, j]))
    for c in range(N):   # Gauss-Jordan with exact pivots
        p = next(r for r in range(c, N) if M[r][c] != 0)
        M[c], M[p] = M[p], M[c]
        inv = 1 / M[c][c]
        M[c] = [x * inv for x in M[c]]
        for r in range(N):
            if r != c and M[r][c] != 0:
                f = M[r][c]
                M[r] = [x - f * y for x, y in zip(M[r], M[c])]
    L = np.zeros((n, n))
    for r, (i, j) in enumerate(unk):
        L[i, j] = float(M[r][N])
    return L


@pytest.mark.parametrize("blk", [[2, 0, 1], [1, 2, 0], [2, 0, 2, 0], [1, 2, 0, 1, 1], [2, 0, 1, 2, 0, 1]])
def test_quasi_solve_matches_exact_brute_force(blk):
    n = len(blk)
    T, E, d = _quasi_problem(n, blk, 7 * n + sum(blk))
    L = oracle.alg2_quasi(T, E, np.array(blk), d)
    ref = _exact_block_solve(T, E, blk)
    assert np.max(np.abs(L - ref)) <= 1e-13 * np.max(np.abs(ref))
    assert np.all(L[~oracle.block_lower_mask(np.array(blk))] == 0)


@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("cap", [0.0, 1e-3])
def test_quasi_solve_with_1x1_blocks_is_alg2(dt, cap):
    n = 40
    rng = np.random.default_rng(5)
    d = np.sort(rng.uniform(0.0, 1.0, n)) + np.arange(n) * 0.01
    T = (np.triu(rng.standard_normal((n, n)) * 0.1, 1) + np.diag(d)).astype(dt)
    E = np.tril(rng.standard_normal((n, n)) * 1e-3, -1).astype(dt)
    L = oracle.alg2_quasi(T, E, np.ones(n, dtype=np.int32), d, cap)
    assert np.array_equal(L, oracle.alg2(T, E, d, cap))


def test_quasi_closed_form_order_3():
    # blocks [2 x 2, 1 x 1]: the one unknown block X = L[2, 0:2] solves
    # t22 X - X T00 = -E[2, 0:2], i.e. X = -E[2, 0:2] (t22 I - T00)^-1
    blk = [2, 0, 1]
    T, E, d = _quasi_problem(3, blk, 11)
    L = oracle.alg2_quasi(T, E, np.array(blk), d)
    X = -E[2, 0:2] @ np.linalg.inv(T[2, 2] * np.eye(2) - T[0:2, 0:2])
    assert np.max(np.abs(L[2, 0:2] - X)) <= 1e-14 * np.max(np.abs(X))


@pytest.mark.parametrize("dt,u", [(np.float64, 2.0 ** -53), (np.float32, 2.0 ** -24)])
def test_quasi_solve_residual_at_size(dt, u):
    n = 200
    rng = np.random.default_rng(2)
    blk = np.ones(n, dtype=np.int32)
    k = 0
    while k < n - 1:
        if rng.uniform() < 0.4:
            blk[k], blk[k + 1] = 2, 0
            k += 2
        else:
            k += 1
    T, E, d = _quasi_problem(n, blk, 3, dt)
    L = oracle.alg2_quasi(T, E, blk, d).astype(np.float64)
    T64, E64 = T.astype(np.float64), E.astype(np.float64)
    mask = oracle.block_lower_mask(blk)
    R = np.where(mask, T64 @ L - L @ T64 + E64, 0.0)
    scale = np.linalg.norm(np.abs(T64) @ np.abs(L) + np.abs(L) @ np.abs(T64)) + np.linalg.norm(E64)
    assert np.linalg.norm(R) <= 20 * u * scale
    assert np.all(L[~mask] == 0)


def test_quasi_shared_eigenvalue_is_rejected():
    # two 2 x 2 blocks with the same complex pair: the block equation between
    # them is singular (the analogue of Theorem 1)
    blk = np.array([2, 0, 2, 0])
    T = np.triu(np.full((4, 4), 0.25), 1)
    for k in (0, 2):
        T[k, k] = T[k + 1, k + 1] = 0.5
        T[k, k + 1], T[k + 1, k] = 0.25, -0.25
    E = np.where(oracle.block_lower_mask(blk), 1.0, 0.0)
    with pytest.raises(oracle.SolveError) as ei:
        oracle.alg2_quasi(T, E, blk, np.diagonal(T).copy())
    assert ei.value.code == oracle.NONDISTINCT


def test_quasi_blocks_read_complex_pairs_only():
    # a 2 x 2 diagonal block with real eigenvalues is split, one with complex
    # eigenvalues kept; rows are taken from the top
    T = np.array([[1.0, 0.5, 0.0, 0.0],
                  [1e-3, 1.2, 0.0, 0.0],      # real pair: (1 - 1.2)^2 + 4 (0.5)(1e-3) > 0
                  [0.0, 0.0, 2.0, 0.4],
                  [0.0, 0.0, -0.3, 2.0]])     # complex pair: 0 + 4 (0.4)(-0.3) < 0
    assert list(oracle.quasi_blocks(T)) == [1, 1, 2, 0]


@pytest.mark.parametrize("n", [64, 300])
def test_quasi_refinement_recovers_planted_form(n):
    p = inputs.quasi_real(n)
    assert (p.blk == 2).sum() > n // 8
    r = oracle.refine(p.A, p.Qhat, lp="f32", quasi=True)
    assert r.status == oracle.OK and r.iters <= 4 and r.hp_gemms == 4 * r.iters
    That = r.Q.T @ p.A @ r.Q
    blk = oracle.quasi_blocks(That)
    assert np.array_equal(blk, p.blk)
    rT, rQ = oracle.residuals_dd(p.A, r.Q, blk=blk)
    tol = oracle.default_tol(n)
    assert rT <= tol and rQ <= tol
    # eigenvalues of the diagonal blocks against the planted ones, row by row
    ev = np.zeros(n, dtype=np.complex128)
    for k in range(n):
        if blk[k] == 2:
            w = np.linalg.eigvals(That[k:k + 2, k:k + 2])
            ev[k], ev[k + 1] = w[np.argmax(w.imag)], w[np.argmin(w.imag)]
        elif blk[k] == 1:
            ev[k] = That[k, k]
    assert np.max(np.abs(ev - p.lam)) <= 1e-12


def test_quasi_form_equals_triangular_form_on_real_spectra():
    # every 2 x 2 diagonal block of T^ has real eigenvalues: the blocks are all
    # 1 x 1 and the two forms take the same steps
    p = inputs.jittered_real(96)
    rq = oracle.refine(p.A, p.Qhat, lp="f32", quasi=True)
    rt = oracle.refine(p.A, p.Qhat, lp="f32")
    assert rq.status == rt.status == oracle.OK and rq.iters == rt.iters
    assert np.array_equal(rq.Q, rt.Q)
