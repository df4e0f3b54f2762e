"""Pins of the double-double target oracle (CPU only).

The oracle of Alg. 4 with hp = double-double and lp = float64
(``oracle.ddtarget``) is checked against exact rational arithmetic (its
double-double product, its 128-bit residuals and sampled entries), against
closed forms (Lemma 2 for the Newton-Schulz step, eq. (NSmerged) for the
update, the divisor of a two-by-two solve), and against the planted truth of
the double-double workload (eigenvalues and Schur vectors of A = Q0 T0 Q0^T).
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import ddtarget as D
from paper_2203_10879_gb300 import inputs

U_DD = 2.0 ** -104


def _dd_random(rng, shape, scale=1.0):
    hi = rng.standard_normal(shape) * scale
    lo = hi * rng.uniform(-1, 1, shape) * 2.0 ** -53
    lo = (hi + lo) - hi            # representable low part below half an ulp of hi
    return np.asfortranarray(hi), np.asfortranarray(lo)


def _exact(x):
    h, l = x
    return [[Fraction(h[i, j]) + Fraction(l[i, j]) for j in range(h.shape[1])] for i in range(h.shape[0])]


def _mat(a, b):
    return [[sum(a[i][k] * b[k][j] for k in range(len(b))) for j in range(len(b[0]))] for i in range(len(a))]


def _t(a):
    return [list(r) for r in zip(*a)]


@pytest.mark.parametrize("m,n,k,transA", [(5, 7, 6, False), (4, 3, 9, True), (1, 1, 1, False)])
def test_gemm_dd_matches_exact_rationals(rng, m, n, k, transA):
    A = _dd_random(rng, (k, m) if transA else (m, k))
    B = _dd_random(rng, (k, n))
    C = D.gemm(A, B, transA=transA)
    Ae, Be = _exact(A), _exact(B)
    Ce = _mat(_t(Ae) if transA else Ae, Be)
    absA = np.abs(A[0].T if transA else A[0])
    bound = 4 * k * U_DD * (absA @ np.abs(B[0]))
    for i in range(m):
        for j in range(n):
            err = abs(Fraction(C[0][i, j]) + Fraction(C[1][i, j]) - Ce[i][j])
            assert float(err) <= bound[i, j], (i, j, float(err), bound[i, j])


def _near_orthogonal_dd(rng, n, eps):
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return (np.asfortranarray(q), np.asfortranarray(eps * rng.standard_normal((n, n))))


def test_residuals_q_match_exact_rationals(rng):
    n = 6
    A = _dd_random(rng, (n, n))
    Q = _near_orthogonal_dd(rng, n, 1e-20)
    rT, rQ = D.residuals_q(A, Q)
    Ae, Qe = _exact(A), _exact(Q)
    M = _mat(_t(Qe), _mat(Ae, Qe))
    G = _mat(_t(Qe), Qe)
    st = sum(float(M[i][j]) ** 2 for i in range(n) for j in range(n) if i > j)
    so = sum(float(G[i][j] - (1 if i == j else 0)) ** 2 for i in range(n) for j in range(n))
    sa = sum(float(Ae[i][j]) ** 2 for i in range(n) for j in range(n))
    assert rT == pytest.approx(math.sqrt(st / sa), rel=1e-12)
    assert rQ == pytest.approx(math.sqrt(so), rel=1e-6)     # r_Q ~ 1e-16 + 1e-20 terms
    assert 1e-18 < rQ < 1e-14


def test_sampled_entries_q_match_exact_rationals(rng):
    n = 7
    A = _dd_random(rng, (n, n))
    Q = _near_orthogonal_dd(rng, n, 1e-22)
    rows = np.array([0, 3, 6, 2, 5])
    cols = np.array([0, 1, 6, 4, 5])
    t, y = D.sample_entries_q(A, Q, rows, cols)
    Ae, Qe = _exact(A), _exact(Q)
    M = _mat(_t(Qe), _mat(Ae, Qe))
    G = _mat(_t(Qe), Qe)
    for s, (i, j) in enumerate(zip(rows, cols)):
        te = M[i][j]
        ye = G[i][j] - (1 if i == j else 0)
        assert abs(float(Fraction(t[0][s]) + Fraction(t[1][s]) - te)) <= 1e-31 * (1 + abs(float(te)))
        assert abs(float(Fraction(y[0][s]) + Fraction(y[1][s]) - ye)) <= 1e-31


def test_alg2_dd_divisors_equal_float64_alg2_without_low_parts(rng):
    n = 40
    T = np.triu(rng.standard_normal((n, n))) + np.diag(np.arange(n) * 0.5)
    E = np.tril(rng.standard_normal((n, n)), -1) * 1e-3
    d = (np.diagonal(T).copy(), np.zeros(n))
    L1 = D.alg2_dd_divisors(T, E, d)
    L2 = oracle.alg2(T, E, np.diagonal(T).copy())
    assert np.array_equal(L1, L2)
    # and the result solves the equation of Sec. 2.1 (Kronecker brute force at n = 6)
    Ts, Es = T[:6, :6], E[:6, :6]
    hi, lo = oracle.kron_solve(Ts, Es)
    Ls = D.alg2_dd_divisors(Ts, Es, (np.diagonal(Ts).copy(), np.zeros(6)))
    assert np.max(np.abs(Ls - (hi + lo))) <= 1e-13 * np.max(np.abs(hi))


def test_alg2_dd_divisor_resolves_equal_float64_diagonal():
    # n = 2: l_21 = -e_21 / (t_22 - t_11); the two diagonal entries coincide in
    # float64 and differ in their low parts, so the divisor is 2^-59.
    T = np.array([[1.0, 0.25], [0.0, 1.0]])
    E = np.array([[0.0, 0.0], [3.0 * 2.0 ** -70, 0.0]])
    d = (np.array([1.0, 1.0]), np.array([-(2.0 ** -60), 2.0 ** -60]))
    L = D.alg2_dd_divisors(T, E, d)
    assert L[1, 0] == -3.0 * 2.0 ** -70 / 2.0 ** -59
    with pytest.raises(oracle.SolveError):
        D.alg2_dd_divisors(T, E, (np.array([1.0, 1.0]), np.zeros(2)))


def test_ns_init_dd_lemma2():
    # Lemma 2: Q^T Q - I = -3/4 Y^2 + 1/4 Y^3 after one Newton-Schulz step, Y = Qhat^T Qhat - I.
    n = 24
    rng = np.random.default_rng(5)
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    Qhat = q @ (np.eye(n) + 1e-5 * rng.standard_normal((n, n)))
    Q, y = D.ns_init_dd(Qhat)
    Y = Qhat.T @ Qhat - np.eye(n)           # float64 is enough for the O(Y^2) right side
    lhs = D.dd_add(D.gemm(Q, Q, transA=True), D.dd_neg(D.dd(np.eye(n))))
    rhs = -0.75 * Y @ Y + 0.25 * Y @ Y @ Y
    diff = (lhs[0] - rhs) + lhs[1]
    assert y == pytest.approx(np.linalg.norm(Qhat.T @ Qhat - np.eye(n)), rel=1e-6)
    assert np.linalg.norm(rhs) > 1e-10
    assert np.linalg.norm(diff) <= 1e-6 * np.linalg.norm(rhs)


def test_merged_update_dd_equals_newton_schulz_of_Q_I_plus_W():
    # eq. (NSmerged): with the full Sigma, 1/2 Q Sigma is one Newton-Schulz step
    # of Q (I + W); the truncated Sigma drops 1/2 Q (W^2 Y + W^2 Y W).
    p = inputs.planted_dd(32, inputs.eig_unit_step(32), 77, pert=1e-4)
    A = (p.A_hi, p.A_lo)
    Q, _ = D.ns_init_dd(p.Qhat)
    Q = D.gemm(Q, D.dd(np.eye(32) + 1e-4 * np.triu(np.ones((32, 32)))))   # make Y visibly nonzero
    parts = {}
    Qf, _ = D.iteration_dd(A, Q, full_sigma=True, parts=parts)
    W = parts["W"]
    Qh = D.gemm(Q, D.dd(np.eye(32) + W))
    G = D.gemm(Qh, Qh, transA=True)
    direct = D.dd_scale(D.gemm(Qh, D.dd_add(D.dd(3.0 * np.eye(32)), D.dd_neg(G))), 0.5)
    diff = (Qf[0] - direct[0]) + (Qf[1] - direct[1])
    Y = D._round(parts["Y"])
    dropped = 0.5 * D._round(Q) @ (W @ W @ Y + W @ W @ Y @ W)
    assert np.linalg.norm(dropped) > 1e-14
    assert np.linalg.norm(diff) <= 1e-3 * np.linalg.norm(dropped)
    Qt, _ = D.iteration_dd(A, Q, full_sigma=False)
    gap = (Qf[0] - Qt[0]) + (Qf[1] - Qt[1])
    assert np.linalg.norm(gap - dropped) <= 1e-3 * np.linalg.norm(dropped)


@pytest.mark.parametrize("n", [64, 100])
def test_refine_dd_recovers_planted_decomposition(n):
    p = inputs.unit_step_dd(n)
    A = (p.A_hi, p.A_lo)
    r = D.refine_dd(A, p.Qhat)
    tol = D.default_tol_dd(n)
    assert r.status == oracle.OK
    assert r.hp_gemms == 4 * r.iters
    rT, rQ = D.residuals_q(A, r.Q)
    assert rT <= tol and rQ <= tol, (rT, rQ, tol)
    T, _ = D.form_residual_dd(A, r.Q)
    dlam = (np.diagonal(T[0]) - p.lam) + np.diagonal(T[1])
    assert np.max(np.abs(dlam)) <= 1e-26
    s = np.sign(np.sum(r.Q[0] * p.Q0_hi, axis=0))
    dq = (r.Q[0] * s - p.Q0_hi) + (r.Q[1] * s - p.Q0_lo)
    assert np.max(np.abs(dq)) <= 1e-25
    # the float64 start is far from the target: the first pass contracts by the
    # float64 solve's relative accuracy, not by the square
    h = [x.r_T for x in r.history]
    assert h[0] > 1e-15
    assert h[1] <= max(10 * h[0] ** 2, 10 * n * 2.0 ** -53 * h[0])


def test_planted_dd_factor_is_orthogonal_to_double_double_accuracy():
    n = 10
    p = inputs.unit_step_dd(n)
    Q = _exact((p.Q0_hi, p.Q0_lo))
    G = _mat(_t(Q), Q)
    off = max(abs(float(G[i][j] - (1 if i == j else 0))) for i in range(n) for j in range(n))
    assert off <= 1e-30
    rT, rQ = D.residuals_q((p.A_hi, p.A_lo), (p.Q0_hi, p.Q0_lo))
    assert rT <= 1e-30 and rQ <= 1e-30
