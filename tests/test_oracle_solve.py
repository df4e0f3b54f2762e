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


# ---------------------------------------------------------------------------
# The divisor reading of the low-precision solves: t_ii - t_jj is formed from
# the high-precision diagonal and rounded once to the low precision. Two
# diagonal entries 1e-9 apart near 1 are equal once rounded to FP32, so a
# divisor formed from the FP32 (or complex64) T would be zero.

def _alg2_f32_py(T32, E32, d):
    """Alg. 2 in FP32, each operation rounded by numpy's float32 scalars, with
    the divisor formed in float64 from ``d`` and rounded once to float32."""
    f = np.float32
    n = T32.shape[0]
    L = np.zeros((n, n), dtype=np.float32)
    for j in range(n - 1):
        for i in range(n - 1, j, -1):
            s1 = f(0.0)
            for k in range(i + 1, n):
                s1 = f(s1 + f(T32[i, k] * L[k, j]))
            s2 = f(0.0)
            for k in range(j):
                s2 = f(s2 + f(L[i, k] * T32[k, j]))
            e = f(f(E32[i, j] + s1) - s2)
            L[i, j] = f(-e / f(float(d[i]) - float(d[j])))
    return L


def _near_equal_pair(n, seed):
    rng = np.random.default_rng(seed)
    d = np.sort(rng.uniform(0.0, 3.0, n))
    d[n // 2] = 1.0
    d[n // 2 + 1] = 1.0 + 1e-9
    assert np.float32(d[n // 2]) == np.float32(d[n // 2 + 1])
    T = np.triu(rng.standard_normal((n, n)) * 0.1, 1) + np.diag(d)
    E = np.tril(rng.standard_normal((n, n)) * 1e-12, -1)
    return T, E, d


def test_alg2_float32_divisor_formed_in_high_precision():
    T, E, d = _near_equal_pair(6, 11)
    T32, E32 = T.astype(np.float32), E.astype(np.float32)
    L = oracle.alg2(T32, E32, d)
    assert L.dtype == np.float32 and np.all(np.isfinite(L))
    # bit for bit the FP32 operations with the divisor rounded once from float64
    assert np.array_equal(L, _alg2_f32_py(T32, E32, d))
    i = 6 // 2 + 1
    assert L[i, i - 1] != 0.0
    # the same solve with divisors formed from the FP32 diagonal hits a zero divisor
    with pytest.raises(oracle.SolveError) as ei:
        oracle.alg2(T32, E32)
    assert ei.value.code == oracle.NONDISTINCT


def test_alg2_complex64_divisor_formed_in_high_precision():
    # n = 2: l_21 = -e_21 / fl32(t_22 - t_11) with a real divisor of 1e-9, so
    # the complex division reduces to the two real ones
    d = np.array([1.0 + 0.25j, 1.0 + 1e-9 + 0.25j])
    assert np.complex64(d[0]) == np.complex64(d[1])
    T = np.array([[d[0], 0.5 - 0.125j], [0.0, d[1]]]).astype(np.complex64)
    E = np.array([[0.0, 0.0], [3e-12 - 2e-12j, 0.0]]).astype(np.complex64)
    L = oracle.alg2(T, E, d)
    den = np.float32(d[1].real - d[0].real)
    assert L.dtype == np.complex64
    assert L[1, 0].real == -E[1, 0].real / den and L[1, 0].imag == -E[1, 0].imag / den
    with pytest.raises(oracle.SolveError) as ei:
        oracle.alg2(T, E)
    assert ei.value.code == oracle.NONDISTINCT
    # a larger case: finite, and equal to the complex128 solve to FP32 accuracy
    Tr, Er, dr = _near_equal_pair(8, 12)
    Tc = (Tr + 0.5j * np.triu(Tr, 1)).astype(np.complex128)
    dc = dr + 0.0j
    np.fill_diagonal(Tc, dc)
    Ec = (Er - 0.5j * Er).astype(np.complex128)
    L64 = oracle.alg2(Tc.astype(np.complex64), Ec.astype(np.complex64), dc)
    L128 = oracle.alg2(Tc, Ec, dc)
    assert np.all(np.isfinite(L64))
    assert np.max(np.abs(L64 - L128)) <= 1e-5 * np.max(np.abs(L128))
