"""Pins of the multi-word oracle (oracle.mptarget: Alg. 4 with an exact
fixed-point high precision and float64 low precision, Sec. 2.4 and Sec. 3's
multi-double working precisions) and of the exact planted recipe it is run on.

Each pin checks the oracle against something other than itself: exact rational
arithmetic (fractions.Fraction) for the conversions, products, residuals and
the Newton-Schulz identity of Sec. 2.3; the exactly known Schur decomposition
of the planted inputs; the double-double oracle (C TwoProd/TwoSum products)
at the double-double tolerance; and the rate of convergence that a float64
correction allows."""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import ddtarget
from oracle import mptarget as mp
from paper_2203_10879_gb300 import inputs

F = mp.FBITS


def _rand_fx(rng, shape, bits=200):
    """Random fixed-point integers of about `bits` bits (values of order 2^(bits - F))."""
    out = np.empty(shape, dtype=object)
    for idx in np.ndindex(shape):
        v = int.from_bytes(rng.bytes(bits // 8 + 1), "little") >> 7
        out[idx] = -v if rng.uniform() < 0.5 else v
    return out


def test_conversions_are_exact():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((7, 5)) * np.exp2(rng.integers(-60, 60, (7, 5)))
    X = mp.to_fx(x)
    for idx in np.ndindex(x.shape):
        assert Fraction(int(X[idx]), 1 << F) == Fraction(float(x[idx]))
    assert np.array_equal(mp.to_float(X), x)


def test_words_are_the_nearest_doubles_of_what_is_left():
    rng = np.random.default_rng(2)
    X = _rand_fx(rng, (40,), bits=240)
    w0, w1, w2 = mp.to_words(X, F, 3)
    for i in range(40):
        r = Fraction(int(X[i]), 1 << F)
        for w in (w0[i], w1[i], w2[i]):
            # nearest: no double on the other side of r is closer
            assert abs(r - Fraction(w)) <= abs(r - Fraction(np.nextafter(w, np.inf)))
            assert abs(r - Fraction(w)) <= abs(r - Fraction(np.nextafter(w, -np.inf)))
            r -= Fraction(w)
        # three words hold the value to 2^-159 relative (two half-ulps of 53 bits each)
        assert abs(r) <= Fraction(abs(int(X[i])), 1 << F) * Fraction(1, 1 << 158)


def test_product_is_the_rounded_exact_product():
    rng = np.random.default_rng(3)
    A, B = _rand_fx(rng, (4, 6)), _rand_fx(rng, (6, 3))
    C = mp.matmul_fx(A, B)
    for i in range(4):
        for j in range(3):
            exact = sum(Fraction(int(A[i, k]), 1 << F) * Fraction(int(B[k, j]), 1 << F) for k in range(6))
            assert abs(Fraction(int(C[i, j]), 1 << F) - exact) <= Fraction(1, 1 << (F + 1))


def test_residuals_against_fractions():
    rng = np.random.default_rng(4)
    n = 5
    A = rng.standard_normal((n, n))
    Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
    rT, rQ = mp.residuals_exact(A, Q)
    Af = [[Fraction(float(v)) for v in row] for row in A]
    Qf = [[Fraction(float(v)) for v in row] for row in Q]
    M = [[sum(Qf[k][i] * Af[k][l] * Qf[l][j] for k in range(n) for l in range(n)) for j in range(n)]
         for i in range(n)]
    G = [[sum(Qf[k][i] * Qf[k][j] for k in range(n)) - (1 if i == j else 0) for j in range(n)] for i in range(n)]
    sE = sum(M[i][j] ** 2 for i in range(n) for j in range(i))
    sA = sum(v ** 2 for row in Af for v in row)
    assert rT == pytest.approx(math.sqrt(sE / sA), rel=1e-15)
    assert rQ == pytest.approx(math.sqrt(sum(v ** 2 for row in G for v in row)), rel=1e-15)


def test_newton_schulz_step_identity():
    # Sec. 2.3: Q1 = 1/2 Q (3I - Q^T Q) satisfies Q1^T Q1 - I = -3/4 Y^2 + 1/4 Y^3
    # with Y = Q^T Q - I, exactly; the oracle's Q1 is rounded to 2^-F
    rng = np.random.default_rng(5)
    n = 6
    Qh = np.linalg.qr(rng.standard_normal((n, n)))[0] + 1e-6 * rng.standard_normal((n, n))
    Q1, y0 = mp.ns_init_fx(Qh)
    Qf = [[Fraction(float(v)) for v in row] for row in Qh]
    Y = [[sum(Qf[k][i] * Qf[k][j] for k in range(n)) - (1 if i == j else 0) for j in range(n)] for i in range(n)]
    mm = lambda X, Z: [[sum(X[i][k] * Z[k][j] for k in range(n)) for j in range(n)] for i in range(n)]
    Y2 = mm(Y, Y)
    Y3 = mm(Y2, Y)
    Q1f = [[Fraction(int(Q1[i, j]), 1 << F) for j in range(n)] for i in range(n)]
    Y1 = [[sum(Q1f[k][i] * Q1f[k][j] for k in range(n)) - (1 if i == j else 0) for j in range(n)] for i in range(n)]
    for i in range(n):
        for j in range(n):
            assert abs(Y1[i][j] - (-Fraction(3, 4) * Y2[i][j] + Fraction(1, 4) * Y3[i][j])) <= Fraction(n, 1 << (F - 4))
    assert y0 == pytest.approx(math.sqrt(float(sum(v * v for row in Y for v in row))), rel=1e-14)


@pytest.mark.parametrize("n", [32, 64])
def test_exact_planted_recipe_is_exact(n):
    p = inputs.unit_step_exact(n)
    Qi = (p.Q0 * n).astype(np.int64).astype(object)
    assert np.array_equal(Qi.astype(float) / n, p.Q0)
    G = np.dot(Qi.T, Qi)
    assert all(G[i, j] == (n * n if i == j else 0) for i in range(n) for j in range(n))
    Ti = (p.T0 * 2 ** 20).astype(np.int64).astype(object)
    assert np.array_equal(Ti.astype(float) / 2 ** 20, p.T0)
    Ae = np.dot(np.dot(Qi, Ti), Qi.T)   # A n^2 2^20, exact
    assert all(Fraction(float(p.A[i, j])) * n * n * 2 ** 20 == Ae[i, j] for i in range(n) for j in range(n))
    assert np.allclose(np.diag(p.T0), p.lam) and np.all(np.tril(p.T0, -1) == 0)


@pytest.mark.parametrize("n", [16, 64])
def test_refinement_recovers_the_exact_schur_form(n):
    p = inputs.unit_step_exact(n)
    r = mp.refine_fx(p.A, p.Qhat)
    assert r.status == 0 and r.iters == 4 and r.hp_gemms == 4 * r.iters
    tol = mp.default_tol_td(n)
    rT, rQ = mp.residuals_exact(p.A, r.Q)
    assert rT <= tol and rQ <= tol
    Q0 = mp.to_fx(p.Q0)
    s = [1 if sum(r.Q[:, j] * Q0[:, j]) > 0 else -1 for j in range(n)]
    err = max(abs(int(r.Q[i, j]) - s[j] * int(Q0[i, j])) for i in range(n) for j in range(n))
    assert err <= 2 ** (F - 170)   # far below the triple-double target
    lam = mp.to_fx(p.lam)
    assert max(abs(int(r.That[i, i]) - int(lam[i])) for i in range(n)) <= 2 ** (F - 170)


def test_float64_correction_limits_the_rate():
    # with the correction L from a float64 solve each pass gains at most a factor
    # near u64 once the error is below u64 (Alg. 4's mixed precision): not the
    # quadratic step of exact arithmetic (which would give ~1e-56 from 5e-28)
    r = mp.refine_fx(inputs.unit_step_exact(64).A, inputs.unit_step_exact(64).Qhat)
    rs = [h.r_T for h in r.history]
    assert rs[1] <= 1e-26 and rs[2] >= 1e-50 and rs[2] <= 1e-40 and rs[2] / rs[1] >= 1e-20


def test_fixed_point_oracle_agrees_with_double_double_oracle():
    # the same Alg. 4 at the double-double tolerance: the passes and the residual
    # measures agree, and the factors differ by far less than their own distance
    # from the exact Schur factors (r_T ~ 5e-28): the double-double rounding of
    # the C oracle's hp products (its orthogonality error is ~3e-31, the fixed
    # point's ~2e-41)
    p = inputs.unit_step_dd(64)
    n = 64
    rd = ddtarget.refine_dd((p.A_hi, p.A_lo), p.Qhat)
    rf = mp.refine_fx((p.A_hi, p.A_lo), p.Qhat, tol=ddtarget.default_tol_dd(n))
    assert rd.status == rf.status == 0 and rd.iters == rf.iters
    assert [h.r_T for h in rd.history] == pytest.approx([h.r_T for h in rf.history], rel=1e-4)
    Qf = mp.to_fx(rd.Q)
    err = max(abs(int(rf.Q[i, j]) - int(Qf[i, j])) for i in range(n) for j in range(n))
    assert err <= 2 ** (F - 92)
    rTd, rQd = mp.residuals_exact((p.A_hi, p.A_lo), Qf)
    rTf, rQf = mp.residuals_exact((p.A_hi, p.A_lo), rf.Q)
    assert rTd == pytest.approx(rTf, rel=1e-4) and rQf < 1e-38 and rQd < 1e-29


def test_six_double_tolerance_is_reached_in_seven_passes():
    # the 100-digit setting of Sec. 3 (six doubles): from a float64 start each
    # pass gains about the factor u64 that the float64 correction allows, so the
    # tolerance 1e-93 n is reached on the seventh pass (the paper reports 7-8
    # iterations for 100 digits), and the factors are the exact planted ones
    F6 = mp.FBITS_D6
    p = inputs.unit_step_exact(16)
    r = mp.refine_fx(p.A, p.Qhat, tol=mp.default_tol_d6(16), F=F6)
    assert r.status == 0 and r.iters == 7 and r.hp_gemms == 28
    rT, rQ = mp.residuals_exact(p.A, r.Q, F=F6)
    assert rT <= mp.default_tol_d6(16) and rQ <= mp.default_tol_d6(16)
    Q0 = mp.to_fx(p.Q0, F6)
    s = [1 if sum(r.Q[:, j] * Q0[:, j]) > 0 else -1 for j in range(16)]
    err = max(abs(int(r.Q[i, j]) - s[j] * int(Q0[i, j])) for i in range(16) for j in range(16))
    assert err <= 2 ** (F6 - 330)
