"""Pins of the oracle's refinement iteration (CPU only).

Alg. 4 and eqs. (NS), (NSmerged) of Sec. 2.4, Lemma 2, Theorem 3, and the
printed product counts of Tables 3/4.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2203_10879_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_ns_identity_lemma2(rng):
    # Lemma 2: Q_new^H Q_new - I = -3/4 Y^2 + 1/4 Y^3 with Y = Qhat^H Qhat - I.
    n = 40
    Q0, _ = np.linalg.qr(rng.standard_normal((n, n)))
    Qhat = Q0 @ (np.eye(n) + 1e-3 * rng.standard_normal((n, n)))
    Y = Qhat.T @ Qhat - np.eye(n)
    Qn, y = oracle.ns_init(Qhat)
    lhs = Qn.T @ Qn - np.eye(n)
    rhs = -0.75 * Y @ Y + 0.25 * Y @ Y @ Y
    assert y == pytest.approx(np.linalg.norm(Y), rel=1e-12)
    assert np.linalg.norm(lhs - rhs) <= 1e-13
    assert np.linalg.norm(rhs) > 1e-6       # the identity is not trivially small here


def test_merged_update_equals_newton_schulz_of_Q_I_plus_W():
    # eq. (NSmerged): with the full Sigma, 1/2 Q Sigma equals one Newton-Schulz
    # step applied to Q (I + W); the truncated Sigma differs by 1/2 Q (W^2 Y + W^2 Y W).
    p = inputs.planted(48, inputs.eig_unit_step(48), 11, pert=3e-3, low="f64")
    Q, _ = oracle.ns_init(p.Qhat)
    Q = Q @ (np.eye(48) + 1e-4 * np.triu(np.ones((48, 48))))   # make Y visibly nonzero
    parts = {}
    Qfull, _ = oracle.iteration(p.A, Q, lp="f64", full_sigma=True, parts=parts)
    W, Y = parts["W"], parts["Y"]
    Qh = Q @ (np.eye(48) + W)
    direct = 0.5 * Qh @ (3 * np.eye(48) - Qh.T @ Qh)
    assert np.linalg.norm(Qfull - direct) <= 1e-13 * np.linalg.norm(direct)
    Qtr, _ = oracle.iteration(p.A, Q, lp="f64", full_sigma=False)
    dropped = 0.5 * Q @ (W @ W @ Y + W @ W @ Y @ W)
    assert np.linalg.norm((Qfull - Qtr) - dropped) <= 1e-3 * np.linalg.norm(dropped) + 1e-15
    assert np.linalg.norm(dropped) > 0


def test_W_is_skew_and_solves_the_linearized_equation():
    p = inputs.unit_step_real(64, low="f64")
    Q, _ = oracle.ns_init(p.Qhat)
    parts = {}
    oracle.iteration(p.A, Q, lp="f64", parts=parts)
    W, L, T, E = parts["W"], parts["L"], parts["T"], parts["E"]
    assert np.array_equal(W, -W.T)
    assert np.all(np.diagonal(W) == 0)
    R = np.tril(E - L @ T + T @ L, -1)     # eq. (linearsystem)
    assert np.linalg.norm(R) <= 1e-13 * np.linalg.norm(E)


@pytest.mark.parametrize("lp", ["f64", "f32"])
def test_planted_recovery(lp):
    p = inputs.unit_step_real(64)
    r = oracle.refine(p.A, p.Qhat, lp=lp)
    assert r.status == oracle.OK
    rT, rQ = oracle.residuals_dd(p.A, r.Q)
    tol = oracle.default_tol(64)
    assert rT <= tol and rQ <= tol
    Tq = r.Q.T @ p.A @ r.Q
    # eigenvalues recovered in order (Qhat fixes the order)
    assert np.max(np.abs(np.diagonal(Tq) - p.lam)) <= 1e-12
    # columns of Q match Q0 up to sign (gaps 1/64 >= 1e-2)
    s = np.sign(np.sum(r.Q * p.Q0, axis=0))
    assert np.max(np.abs(r.Q - p.Q0 * s)) <= 1e-12


def test_quadratic_convergence_uniform_precision():
    # Theorem 3: ||stril|| goes to O(eps^2), ||Q^H Q - I|| to O(eps^4).
    p = inputs.planted(64, inputs.eig_unit_step(64), inputs.BASE_SEED + 1, pert=1e-4, low="f64")
    r = oracle.refine(p.A, p.Qhat, lp="f64", max_iter=6)
    h = [x.r_T for x in r.history]
    assert r.status == oracle.OK
    assert h[1] <= 10 * h[0] ** 2 * 64 and h[2] <= 10 * h[1] ** 2 * 64 * 100
    # a linearly convergent iteration at rate 1e-2 would violate the first bound
    assert h[1] < 1e-2 * h[0] * 1e-1
    # orthogonality after the initial Newton-Schulz step ~ 3/4 ||Y0||^2 (+ rounding)
    assert r.history[0].y_norm <= 0.75 * r.y0 ** 2 + 1e-13


def _golden_counts():
    rows = []
    with open(os.path.join(GOLDEN, "matmul_counts.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                it, mm = line.split()
                rows.append((int(it), int(mm)))
    return rows


@pytest.mark.parametrize("pert,want_iters", [(1e-6, 3), (1e-4, 4), (3e-3, 5)])
def test_hp_product_count_matches_tables_3_and_4(pert, want_iters):
    table = dict(_golden_counts())
    p = inputs.planted(64, inputs.eig_unit_step(64), inputs.BASE_SEED + 1, pert=pert, low="f64")
    r = oracle.refine(p.A, p.Qhat, lp="f64", max_iter=10)
    assert r.status == oracle.OK
    assert r.iters == want_iters
    assert r.hp_gemms == table[r.iters]


def test_mixed_precision_converges_like_double():
    p = inputs.jittered_real(256)
    r32 = oracle.refine(p.A, p.Qhat, lp="f32")
    r64 = oracle.refine(p.A, p.Qhat, lp="f64")
    assert r32.status == r64.status == oracle.OK
    assert abs(r32.iters - r64.iters) <= 1
    rT, rQ = oracle.residuals_dd(p.A, r32.Q)
    assert rT <= oracle.default_tol(256) and rQ <= oracle.default_tol(256)


def test_complex_refinement():
    p = inputs.ring_complex(96)
    r = oracle.refine(p.A, p.Qhat, lp="f32")
    assert r.status == oracle.OK
    rT, rQ = oracle.residuals_dd(p.A, r.Q)
    assert rT <= oracle.default_tol(96) and rQ <= oracle.default_tol(96)
    d = np.diagonal(r.Q.conj().T @ p.A @ r.Q)
    assert np.max(np.abs(d - p.lam)) <= 1e-12


def test_failure_path_returns_status():
    # Upper-triangle standard deviation 1/sqrt(n) on a spectrum packed at ~1/n:
    # the triangular equation is too ill-conditioned, the iteration blows up
    # (as in Example 3) and must report it instead of looping.
    p = inputs.jittered_real(128, upper_std=1 / math.sqrt(128))
    r = oracle.refine(p.A, p.Qhat, lp="f32", max_iter=10)
    assert r.status in (oracle.NONFINITE, oracle.NOT_CONVERGED)
    assert r.iters <= 10


def _exact_residuals(A, Q):
    n = A.shape[0]
    Af = [[Fraction(float(A[i, j])) for j in range(n)] for i in range(n)]
    Qf = [[Fraction(float(Q[i, j])) for j in range(n)] for i in range(n)]
    AQ = [[sum(Af[i][k] * Qf[k][j] for k in range(n)) for j in range(n)] for i in range(n)]
    st = Fraction(0)
    so = Fraction(0)
    for i in range(n):
        for j in range(n):
            t = sum(Qf[k][i] * AQ[k][j] for k in range(n))
            if i > j:
                st += t * t
            g = sum(Qf[k][i] * Qf[k][j] for k in range(n)) - (1 if i == j else 0)
            so += g * g
    sa = sum(Af[i][j] ** 2 for i in range(n) for j in range(n))
    return math.sqrt(st / sa), math.sqrt(so)


def test_residuals_dd_match_exact_rational_arithmetic():
    p = inputs.unit_step_real(6, low="f64")
    r = oracle.refine(p.A, p.Qhat, lp="f64")
    Q = r.Q
    rT, rQ = oracle.residuals_dd(p.A, Q)
    eT, eQ = _exact_residuals(p.A, Q)
    assert rT == pytest.approx(eT, rel=1e-12)
    assert rQ == pytest.approx(eQ, rel=1e-12)
    assert eT < 1e-15


def test_sample_entries_dd_match_exact():
    p = inputs.unit_step_real(5, low="f64")
    Q, _ = oracle.ns_init(p.Qhat)
    rows, cols = [4, 2, 0, 3], [0, 1, 0, 3]
    t, y = oracle.sample_entries_dd(p.A, Q, rows, cols)
    n = 5
    Af = [[Fraction(float(p.A[i, j])) for j in range(n)] for i in range(n)]
    Qf = [[Fraction(float(Q[i, j])) for j in range(n)] for i in range(n)]
    for s, (i, j) in enumerate(zip(rows, cols)):
        tij = sum(Qf[l][i] * sum(Af[l][k] * Qf[k][j] for k in range(n)) for l in range(n))
        yij = sum(Qf[l][i] * Qf[l][j] for l in range(n)) - (1 if i == j else 0)
        assert t[s] == pytest.approx(float(tij), rel=1e-14, abs=1e-30)
        assert y[s] == pytest.approx(float(yij), rel=1e-12, abs=1e-31)


def test_sample_entries_dd_complex_match_exact():
    # Gaussian-rational arithmetic: each complex entry as a pair of Fractions
    p = inputs.ring_complex(5)
    Q, _ = oracle.ns_init(p.Qhat)
    rows, cols = [4, 2, 0, 3, 1], [0, 1, 0, 3, 4]
    t, y = oracle.sample_entries_dd(p.A, Q, rows, cols)
    n = 5

    def fr(z):
        return (Fraction(float(z.real)), Fraction(float(z.imag)))

    def mul(a, b):
        return (a[0] * b[0] - a[1] * b[1], a[0] * b[1] + a[1] * b[0])

    def add(a, b):
        return (a[0] + b[0], a[1] + b[1])

    zero = (Fraction(0), Fraction(0))
    Af = [[fr(p.A[i, j]) for j in range(n)] for i in range(n)]
    Qf = [[fr(Q[i, j]) for j in range(n)] for i in range(n)]
    Qc = [[(q[0], -q[1]) for q in row] for row in Qf]
    for s, (i, j) in enumerate(zip(rows, cols)):
        tij = zero
        for l in range(n):
            aq = zero
            for k in range(n):
                aq = add(aq, mul(Af[l][k], Qf[k][j]))
            tij = add(tij, mul(Qc[l][i], aq))
        yij = zero
        for l in range(n):
            yij = add(yij, mul(Qc[l][i], Qf[l][j]))
        if i == j:
            yij = (yij[0] - 1, yij[1])
        assert abs(t[s] - complex(float(tij[0]), float(tij[1]))) <= 1e-15 * max(1.0, abs(t[s]))
        assert abs(y[s] - complex(float(yij[0]), float(yij[1]))) <= 1e-30 + 1e-12 * abs(y[s])


def test_gemm_dd_matches_exact(rng):
    n = 7
    A = rng.standard_normal((n, n))
    B = rng.standard_normal((n, n))
    Bl = B * 1e-17
    Ch, Cl = oracle.gemm_dd(A, None, B, Bl, transA=True)
    for i in range(n):
        for j in range(n):
            ex = sum(Fraction(A[k, i]) * (Fraction(B[k, j]) + Fraction(Bl[k, j])) for k in range(n))
            got = Fraction(Ch[i, j]) + Fraction(Cl[i, j])
            assert abs(float(got - ex)) <= 1e-30 * max(1.0, abs(float(ex)))


@pytest.mark.parametrize("n,passes", [(64, 5), (512, 3)])
def test_variance_reading_of_upper_entries_converges_on_unit_step(n, passes):
    # "N(0, 1/n)" read as variance 1/n (standard deviation 1/sqrt(n)) on the
    # unit-step spectrum (gap 1/64): T0 is then strongly non-normal (strictly
    # upper entries of 0.125 against the gap 1/64 at n = 64), and the mixed
    # iteration still converges to the FP64 target, in 5 passes at n = 64
    p = inputs.unit_step_real(n, upper_std=1.0 / math.sqrt(n))
    r = oracle.refine(p.A, p.Qhat, lp="f32")
    assert r.status == oracle.OK and r.iters == passes
    rT, rQ = oracle.residuals_dd(p.A, r.Q)
    tol = oracle.default_tol(n)
    assert rT <= tol and rQ <= tol
