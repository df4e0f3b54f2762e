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


# ---------------------------------------------------------------------------
# Hermitian A (Sec. 2.5 for complex data): the Schur form is real diagonal, so
# the divisor comes from the real parts of the diagonal

def _herm_problem(n, seed, dt):
    rng = np.random.default_rng(seed)
    d = np.sort(rng.uniform(-1.0, 1.0, n)) + 0j
    E = np.tril(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)), -1) * 1e-4
    return d, E.astype(dt)


@pytest.mark.parametrize("dt", [np.complex64, np.complex128])
def test_hermitian_sym_solve_equals_alg2_with_diagonal_T(dt):
    # the C loops of Alg. 2 in complex arithmetic with a real diagonal T: the
    # same solution up to the rounding of their complex division
    n = 24
    d, E = _herm_problem(n, 31, dt)
    L = oracle.sym_solve(E, d)
    L2 = oracle.alg2(np.diag(d).astype(dt), E, d)
    assert L.dtype == dt
    u = 2.0 ** -24 if dt == np.complex64 else 2.0 ** -53
    assert np.max(np.abs(L - L2)) <= 4 * u * np.max(np.abs(L))


def test_hermitian_sym_solve_satisfies_the_equation():
    n = 40
    d, E = _herm_problem(n, 8, np.complex128)
    L = oracle.sym_solve(E, d)
    T = np.diag(d)
    R = np.tril(T @ L - L @ T, -1) + E
    # rounding: one division per part in sym_solve, complex products and a difference here
    a = np.abs(d)
    bound = 8 * 2.0 ** -53 * ((a[:, None] + a[None, :]) * np.abs(L) + np.abs(E))
    assert np.all(np.tril(np.abs(R), -1) <= np.tril(bound, -1))
    i, j = 7, 3
    assert L[i, j] == -E[i, j].real / (d[i].real - d[j].real) - 1j * E[i, j].imag / (d[i].real - d[j].real)


@pytest.mark.parametrize("n", [64, 200])
def test_hermitian_refinement_matches_eigh(n):
    p = inputs.hermitian_complex(n)
    assert np.array_equal(p.A, p.A.conj().T)
    r = oracle.refine(p.A, p.Qhat, lp="f32", symmetric=True)
    assert r.status == oracle.OK and r.iters <= 4
    w, V = np.linalg.eigh(p.A)
    D = np.diagonal(r.Q.conj().T @ p.A @ r.Q)
    assert np.max(np.abs(D - w)) <= 1e-13
    c = np.sum(np.conj(r.Q) * V, axis=0)
    Qa = r.Q * (c / np.abs(c))
    assert np.max(np.abs(Qa - V)) <= 1e-10
    rT, rQ = oracle.residuals_dd(p.A, r.Q)
    tol = oracle.default_tol(n)
    assert rT <= tol and rQ <= tol
