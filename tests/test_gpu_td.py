"""GPU parity of the triple-double target (hp = three doubles, about 159 bits;
lp = FP64; Sec. 3's multi-double working precisions), through the C ABI,
against the fixed-point oracle (oracle.mptarget) and against planted inputs
whose Schur decomposition is exact (inputs.planted_exact).

Tolerances:
  * product: the residue form with 48 moduli holds each row of op(A) and each
    column of B as integers of t bits (t = 162 for K <= 4096) relative to the
    vector's largest entry, so each entry of the product is within
    K 2^-t max|a_i| max|b_j| of the exact product of the given operands (the
    exact sums of their planes), and within 2^-159 of itself after its one
    rounding to three words; the bound used is (K + 4) 2^-158 max|a_i| max|b_j|;
  * refined factors: exact residuals <= 1e-45 n (the stop test's tolerance);
    Q within 1e-42 of the exact planted Q0 and of the oracle's factor, up to
    column signs, and the diagonal of T^ within 1e-42 ||A||_F of the planted
    eigenvalues (the gap is 1/64: an error of the factors near r_T ~ 1e-47 moves
    them by about 64 r_T ||A||).
"""
import numpy as np
import pytest

from oracle import mptarget as mp
from paper_2203_10879_gb300 import _binding as B
from paper_2203_10879_gb300 import inputs
from gpu_util import from_dev, to_dev

pytestmark = pytest.mark.gpu
F = mp.FBITS


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    B.lib()
    return torch


def _opts(**kw):
    base = dict(target=B.SR_TARGET_TD, lp=B.SR_LP_FP64, qhat_type=B.SR_QHAT_FP64, hp_gemm=B.SR_HP_OZAKI_CRT)
    base.update(kw)
    return B.default_options(**base)


def _handle(n_max, **kw):
    s, h = B.schur_refine_create(n_max, _opts(**kw), None)
    assert s == B.SR_OK, B.status_string(s)
    return h


def _td_dev(planes):
    return to_dev(np.hstack(planes))


def _td_host(t):
    a = from_dev(t)
    c = a.shape[1] // 3
    return a[:, :c], a[:, c:2 * c], a[:, 2 * c:]


def _td_empty(torch, n, c):
    return torch.zeros((3 * c, n), dtype=torch.float64, device="cuda").t()


def _ulp(x):
    return np.abs(np.nextafter(x, np.inf) - x)


def test_td_options_gate(torch):
    bad = [dict(hp_gemm=B.SR_HP_FP64), dict(hp_gemm=B.SR_HP_OZAKI_BF16), dict(lp=B.SR_LP_FP32),
           dict(qhat_type=B.SR_QHAT_FP32), dict(dtype=B.SR_COMPLEX), dict(graph=1)]
    for kw in bad:
        s, h = B.schur_refine_create(64, _opts(**kw), None)
        assert s == B.SR_ERR_UNSUPPORTED and not h.value, kw
    s, h = B.schur_refine_create(64, _opts(ozaki_slices=32), None)
    assert s == B.SR_ERR_INVALID_ARG and not h.value
    s, h = B.schur_refine_create(64, _opts(ozaki_slices=48), None)
    assert s == B.SR_OK
    B.schur_refine_destroy(h)


def _td_random(rng, rows, cols, spread=20):
    """Three planes x0 + x1 + x2 with row scales 2^U(-spread, spread)."""
    sc = np.exp2(rng.integers(-spread, spread + 1, (rows, 1))).astype(float)
    x0 = rng.standard_normal((rows, cols)) * sc
    x1 = x0 * rng.uniform(-1, 1, (rows, cols)) * 2.0 ** -54
    x2 = x1 * rng.uniform(-1, 1, (rows, cols)) * 2.0 ** -54
    return np.asfortranarray(x0), np.asfortranarray(x1), np.asfortranarray(x2)


@pytest.mark.parametrize("m,n,k,transA", [(64, 64, 64, 0), (100, 37, 300, 0), (129, 65, 300, 1), (33, 200, 129, 1)])
def test_td_product_matches_exact_product(torch, m, n, k, transA):
    rng = np.random.default_rng(m * 7 + n + k)
    A = _td_random(rng, k if transA else m, m if transA else k)
    Bm = _td_random(rng, n, k)
    Bm = tuple(np.asfortranarray(p.T) for p in Bm)                     # columns with their own scales
    h = _handle(max(m, n, k))
    try:
        C = _td_empty(torch, m, n)
        s = B.schur_refine_gemm(h, transA, m, n, k, _td_dev(A), _td_dev(Bm), C)
        assert s == B.SR_OK, B.status_string(s)
        c0, c1, c2 = _td_host(C)
    finally:
        B.schur_refine_destroy(h)
    Af = mp.to_fx(A)
    Af = Af.T if transA else Af
    Bf = mp.to_fx(Bm)
    exact = np.dot(Af, Bf)                                             # scale 2^-2F
    got = mp.to_fx((c0, c1, c2)) * (1 << F)                              # scale 2^-2F
    amax = np.abs(A[0].T if transA else A[0]).max(axis=1)
    bmax = np.abs(Bm[0]).max(axis=0)
    for i in range(m):
        for j in range(n):
            bound = (k + 4) * 2.0 ** -158 * amax[i] * bmax[j] * 2.0
            assert abs(int(got[i, j]) - int(exact[i, j])) <= mp._f2i(bound, 2 * F), (i, j)
    # three words, each at most half an ulp of the one before
    nz = c0 != 0
    assert np.all(np.abs(c1[nz]) <= _ulp(c0[nz]) / 2)
    nz1 = c1 != 0
    assert np.all(np.abs(c2[nz1]) <= _ulp(c1[nz1]) / 2)


def _refine(p, torch):
    n = p.n
    h = _handle(n)
    try:
        A = _td_dev((p.A, np.zeros_like(p.A), np.zeros_like(p.A)))
        Q = _td_empty(torch, n, n)
        T = _td_empty(torch, n, n)
        st, nr = B.schur_refine_step(h, n, A, Q, to_dev(p.Qhat), T)
        rs, rT, rQ = B.schur_refine_residuals(h, n, A, Q)
        assert rs == B.SR_OK
        return st, nr, _td_host(Q), _td_host(T), (rT, rQ)
    finally:
        B.schur_refine_destroy(h)


def _sign_fix(Qw, Q0):
    s = np.sign(np.sum(Qw[0] * Q0, axis=0))
    s[s == 0] = 1.0
    return s


def _max_diff_words(Xw, Y, scale=None):
    """max |(x0 + x1 + x2) - Y| in float64: x0 - Y is exact (Sterbenz) and each
    later word nearly cancels what is left, so the sums are exact or within an
    ulp of a number far below the tolerances."""
    d = ((Xw[0] - Y) + Xw[1]) + Xw[2]
    return np.max(np.abs(d))


@pytest.mark.parametrize("n", [32, 64])
def test_td_refinement_matches_oracle(torch, n):
    p = inputs.unit_step_exact(n)
    st, nr, Qw, Tw, (rT, rQ) = _refine(p, torch)
    ref = mp.refine_fx(p.A, p.Qhat)
    assert ref.status == 0 and st == B.SR_OK, B.status_string(st)
    assert nr.iters == ref.iters and nr.hp_gemms == 4 * nr.iters
    tol = mp.default_tol_td(n)
    cT, cQ = mp.residuals_exact(p.A, Qw)
    assert cT <= tol and cQ <= tol
    # the library's own residuals come from its triple-double products: operands
    # cut to 162 bits per vector and results rounded to 159, so near convergence
    # they agree with the exact ones to that floor (about n 2^-159), far below tol
    assert abs(rQ - cQ) <= n * 1e-48 and rQ <= tol
    assert abs(rT - cT) <= n * 1e-47 and rT <= tol
    s = _sign_fix(Qw, p.Q0)
    assert _max_diff_words(Qw, p.Q0 * s) <= 1e-42
    Qo = mp.to_words(ref.Q, F, 3)
    so = _sign_fix(Qo, p.Q0)
    assert np.array_equal(s, so)
    d = mp.to_fx(Qw) - mp.to_fx(Qo)
    assert max(abs(int(v)) for v in d.ravel()) <= mp._f2i(1e-42, F)
    dT = _max_diff_words(tuple(np.diag(t) for t in Tw), p.lam)
    assert dT <= 1e-42 * np.linalg.norm(p.A)


def test_td_workload_full_size(torch):
    # the triple-double workload itself (n = 2048, lambda_k = 1 + k/64): the
    # refined factors against the exact Q0 and T0 over every entry
    p = inputs.unit_step_exact(2048)
    st, nr, Qw, Tw, (rT, rQ) = _refine(p, torch)
    assert st == B.SR_OK, B.status_string(st)
    assert nr.iters == 4 and nr.hp_gemms == 16
    tol = mp.default_tol_td(2048)
    assert rT <= tol and rQ <= tol
    s = _sign_fix(Qw, p.Q0)
    assert _max_diff_words(Qw, p.Q0 * s) <= 1e-42
    anorm = np.linalg.norm(p.A)
    assert _max_diff_words(tuple(np.diag(t) for t in Tw), p.lam) <= 1e-42 * anorm
    assert np.max(np.abs(np.tril(Tw[0], -1))) <= tol * anorm
    # upper triangle of T^ against T0 up to the column signs: T^ = S T0 S
    Tu = tuple(np.triu(t, 1) for t in Tw)
    assert _max_diff_words(Tu, np.triu(p.T0, 1) * np.outer(s, s)) <= 1e-40 * anorm
