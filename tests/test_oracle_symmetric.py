"""Oracle pins for Sec. 2.5 (real symmetric A): the elementwise solve and the
refinement built on it, checked against an independent implementation of
the same equation (the C Alg. 2 with a diagonal T), against the equation
itself, and against LAPACK's symmetric eigensolver (numpy.linalg.eigh)."""
import numpy as np
import pytest

import oracle
from paper_2203_10879_gb300 import inputs
from gpu_util import sign_align


def _sym_problem(n, seed, dt):
    rng = np.random.default_rng(seed)
    d = np.sort(rng.uniform(-1.0, 1.0, n))
    E = np.tril(rng.standard_normal((n, n)) * 1e-4, -1)
    return d, E.astype(dt)


@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("n", [1, 2, 17, 64])
def test_sym_solve_equals_alg2_with_diagonal_T(n, dt):
    d, E = _sym_problem(n, 100 + n, dt)
    L = oracle.sym_solve(E, d)
    L2 = oracle.alg2(np.diag(d).astype(dt), E, d)   # C loops of Alg. 2, off-diagonal T zero
    assert L.dtype == dt
    assert np.array_equal(L, L2)


def test_sym_solve_satisfies_the_equation():
    n = 40
    d, E = _sym_problem(n, 7, np.float64)
    L = oracle.sym_solve(E, d)
    T = np.diag(d)
    R = np.tril(T @ L - L @ T, -1) + E        # stril(TL - LT) = -E (eq. linearsystem)
    # rounding: one division in sym_solve, two products and a difference here
    bound = 4 * 2.0 ** -53 * (np.abs(d)[:, None] + np.abs(d)[None, :]) * np.abs(L) + 2 * 2.0 ** -53 * np.abs(E)
    assert np.all(np.tril(np.abs(R), -1) <= np.tril(bound, -1))
    assert np.all(np.triu(L) == 0)
    # the sign of eq. (lij): l_ij = -e_ij / (t_ii - t_jj)
    i, j = 5, 2
    assert L[i, j] == pytest.approx(-E[i, j] / (d[i] - d[j]), rel=1e-15)


def test_sym_solve_reports_equal_diagonal():
    d = np.array([1.0, 2.0, 1.0])
    E = np.tril(np.ones((3, 3)), -1)
    with pytest.raises(oracle.SolveError) as e:
        oracle.sym_solve(E, d)
    assert e.value.code == oracle.NONDISTINCT


@pytest.mark.parametrize("n", [64, 200])
def test_symmetric_refinement_matches_eigh(n):
    p = inputs.symmetric_real(n)
    assert np.array_equal(p.A, p.A.T)
    r = oracle.refine(p.A, p.Qhat, lp="f32", symmetric=True)
    assert r.status == oracle.OK and r.iters <= 4
    w, V = np.linalg.eigh(p.A)                          # ascending, like lambda
    D = np.diagonal(r.Q.T @ p.A @ r.Q)
    assert np.max(np.abs(D - w)) <= 1e-13
    assert np.max(np.abs(sign_align(r.Q, V) - V)) <= 1e-10
    rT, rQ = oracle.residuals_dd(p.A, r.Q)
    tol = oracle.default_tol(n)
    assert rT <= tol and rQ <= tol


def test_symmetric_and_general_forms_agree_on_symmetric_input():
    p = inputs.symmetric_real(96)
    rs = oracle.refine(p.A, p.Qhat, lp="f32", symmetric=True)
    rg = oracle.refine(p.A, p.Qhat, lp="f32")
    assert rs.status == oracle.OK and rg.status == oracle.OK
    assert np.max(np.abs(sign_align(rs.Q, rg.Q) - rg.Q)) <= 1e-11
