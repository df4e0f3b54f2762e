"""Oracle pins for the entry threshold of Example 4 (Sec. 3): while L is
computed, an entry larger than the threshold in modulus is set to zero at
once, before the entries computed after it use it. Checked against Alg. 2
written out in plain Python floats (the same operations in the same order,
so equal bit for bit), and for the properties the trick fixes."""
import numpy as np
import pytest

import oracle


def _alg2_py(T, E, d, cap):
    """Alg. 2 with the threshold, in Python floats: column j = 0, 1, ..., rows
    i = n-1 down to j+1, l_ij = -(e_ij + sum_{k>i} t_ik l_kj - sum_{k<j} l_ik t_kj)
    / (t_ii - t_jj)."""
    n = T.shape[0]
    L = [[0.0] * n for _ in range(n)]
    for j in range(n - 1):
        for i in range(n - 1, j, -1):
            s1 = 0.0
            for k in range(i + 1, n):
                s1 += float(T[i, k]) * L[k][j]
            s2 = 0.0
            for k in range(j):
                s2 += L[i][k] * float(T[k, j])
            e = float(E[i, j]) + s1 - s2
            l = -e / (float(d[i]) - float(d[j]))
            if cap > 0 and abs(l) > cap:
                l = 0.0
            L[i][j] = l
    return np.array(L)


def _problem(n, seed):
    rng = np.random.default_rng(seed)
    d = np.sort(rng.uniform(0.0, 1.0, n))
    d[n // 2] = d[n // 2 - 1] + 1e-7           # a close pair: large entries in its rows and columns
    T = np.triu(rng.standard_normal((n, n)) * 0.1, 1) + np.diag(d)
    E = np.tril(rng.standard_normal((n, n)) * 1e-6, -1)
    return T, E, d


@pytest.mark.parametrize("cap", [0.0, 1e-5, 1e-3])
@pytest.mark.parametrize("n", [2, 5, 12])
def test_capped_alg2_equals_plain_python(n, cap):
    T, E, d = _problem(n, 31 * n)
    L = oracle.alg2(T, E, d, cap)
    ref = _alg2_py(T, E, d, cap)
    assert np.array_equal(L, ref)


def test_cap_clamps_and_changes_only_what_depends_on_clamped_entries():
    n = 12
    T, E, d = _problem(n, 5)
    L0 = oracle.alg2(T, E, d)
    L1 = oracle.alg2(T, E, d, 1e-5)
    assert np.max(np.abs(L0)) > 1e-5              # the close pair makes some entries large
    assert np.all(np.abs(L1) <= 1e-5)
    big = np.abs(L0) > 1e-5
    # the entries of column 0 computed before the first clamped one are unchanged
    i_first = max(i for i in range(n) if big[i, 0]) if big[:, 0].any() else -1
    for i in range(n - 1, i_first, -1):
        if i > 0:
            assert L1[i, 0] == L0[i, 0]


def test_cap_in_float32_compares_in_float32():
    n = 6
    T, E, d = _problem(n, 9)
    L = oracle.alg2(T.astype(np.float32), E.astype(np.float32), d, 1e-5)
    assert L.dtype == np.float32
    assert np.all(np.abs(L) <= np.float32(1e-5))


def test_symmetric_cap():
    rng = np.random.default_rng(3)
    d = np.array([0.0, 1e-9, 1.0, 2.0])
    E = np.tril(rng.standard_normal((4, 4)) * 1e-6, -1)
    L = oracle.sym_solve(E, d, 1e-5)
    assert L[1, 0] == 0.0                         # -e/1e-9 ~ 1e-3 > cap
    assert L[2, 0] == -E[2, 0] / (d[2] - d[0])
