"""Pins of the oracle's triangular-equation solvers (CPU only).

stril(T L - L T) = -E, Sec. 2.1. Alg. 2 is pinned against a brute-force dense
solve of the operator's matrix in 128-bit arithmetic, against closed forms
(n = 2, diagonal T), against Theorem 1, and by its residual at larger n. Alg. 3
(a different admissible order) is pinned against Alg. 2.
"""
import numpy as np
import pytest

import oracle


def _problem(rng, n, spread=1.0, off=0.3, cplx=False):
    d = np.sort(rng.uniform(0.0, spread, n)) + np.arange(n) * (spread / n)
    T = np.triu(rng.standard_normal((n, n)) * off, 1) + np.diag(d)
    E = np.tril(rng.standard_normal((n, n)), -1)
    if cplx:
        T = T + 1j * (np.triu(rng.standard_normal((n, n)) * off, 1) + np.diag(rng.uniform(0, 0.1, n)))
        E = E + 1j * np.tril(rng.standard_normal((n, n)), -1)
    return np.asfortranarray(T), np.asfortranarray(E)


def _stril(M):
    return np.tril(M, -1)


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 7, 8])
def test_alg2_matches_kronecker_brute_force(rng, n):
    T, E = _problem(rng, n)
    hi, lo = oracle.kron_solve(T, E)
    L = oracle.alg2(T, E)
    scale = np.max(np.abs(hi))
    # the brute force is exact to ~1e-33; Alg. 2 in double has rounding error only
    assert np.max(np.abs(L - hi)) <= 1e-13 * scale
    assert np.all(L[np.triu_indices(n)] == 0.0)


def test_kronecker_solution_satisfies_equation(rng):
    T, E = _problem(rng, 6)
    hi, lo = oracle.kron_solve(T, E)
    R = _stril(T @ hi - hi @ T) + E
    assert np.max(np.abs(R)) <= 1e-14 * np.max(np.abs(E))


def test_alg2_n2_closed_form():
    T = np.array([[0.3, 1.7], [0.0, -1.1]], order="F")
    E = np.array([[0.0, 0.0], [0.25, 0.0]], order="F")
    L = oracle.alg2(T, E)
    assert L[1, 0] == pytest.approx(-0.25 / (-1.1 - 0.3), rel=1e-15)


@pytest.mark.parametrize("cplx", [False, True])
def test_alg2_diagonal_T_closed_form(rng, cplx):
    # eq. (lij) with diagonal T: l_ij = -e_ij / (t_ii - t_jj); the symmetric
    # section writes the same formula without the minus sign, which eq. (lij)
    # and Alg. 2 contradict.
    n = 9
    d = np.arange(n) + rng.uniform(0, 0.5, n)
    if cplx:
        d = d + 1j * rng.uniform(0, 1, n)
    T = np.asfortranarray(np.diag(d))
    E = np.asfortranarray(np.tril(rng.standard_normal((n, n)), -1).astype(T.dtype))
    L = oracle.alg2(T, E)
    want = np.zeros_like(E)
    for j in range(n):
        for i in range(j + 1, n):
            want[i, j] = -E[i, j] / (d[i] - d[j])
    assert np.max(np.abs(L - want)) <= 1e-15 * np.max(np.abs(want))


@pytest.mark.parametrize("n,cplx", [(64, False), (129, False), (77, True)])
def test_alg2_residual_small_at_any_size(rng, n, cplx):
    T, E = _problem(rng, n, spread=4.0, off=0.05, cplx=cplx)
    L = oracle.alg2(T, E)
    R = _stril(T @ L - L @ T) + E
    bound = 10 * n * np.finfo(float).eps * (np.linalg.norm(T) * np.linalg.norm(L) + np.linalg.norm(E))
    assert np.linalg.norm(R) <= bound


def test_alg2_complex_reduces_to_real(rng):
    T, E = _problem(rng, 17)
    Lr = oracle.alg2(T, E)
    Lc = oracle.alg2(T.astype(np.complex128), E.astype(np.complex128))
    assert np.max(np.abs(Lc.imag)) == 0.0
    assert np.max(np.abs(Lc.real - Lr)) <= 1e-15 * np.max(np.abs(Lr))


def test_alg2_float32_tracks_float64(rng):
    T, E = _problem(rng, 48, spread=4.0, off=0.05)
    L64 = oracle.alg2(T, E)
    L32 = oracle.alg2(T.astype(np.float32), E.astype(np.float32), np.diagonal(T).copy())
    assert L32.dtype == np.float32
    err = np.linalg.norm(L32 - L64) / np.linalg.norm(L64)
    assert 1e-9 < err < 1e-5   # single-precision accuracy, not double


def test_thm1_equal_diagonal_is_rejected(rng):
    T, E = _problem(rng, 6)
    T[4, 4] = T[1, 1]
    with pytest.raises(oracle.SolveError) as ei:
        oracle.alg2(T, E)
    assert ei.value.code == oracle.NONDISTINCT
    with pytest.raises(oracle.SolveError):
        oracle.kron_solve(T, E)


@pytest.mark.parametrize("n,nmin", [(16, 2), (37, 2), (37, 5), (64, 8), (33, 40)])
def test_alg3_matches_alg2(rng, n, nmin):
    T, E = _problem(rng, n, spread=4.0, off=0.1)
    L2 = oracle.alg2(T, E)
    L3 = oracle.alg3(T, E, nmin=nmin)
    assert np.max(np.abs(L3 - L2)) <= 1e-12 * np.max(np.abs(L2))


def test_alg3_matches_kronecker(rng):
    T, E = _problem(rng, 8)
    hi, _ = oracle.kron_solve(T, E)
    L3 = oracle.alg3(T, E, nmin=2)
    assert np.max(np.abs(L3 - hi)) <= 1e-13 * np.max(np.abs(hi))
