"""GPU parity of the six-double target (hp = six doubles, about 318 bits: the
100-digit precision of Sec. 3; lp = FP64), through the C ABI, against the
fixed-point oracle (oracle.mptarget with 512 fraction bits) and against planted
inputs whose Schur decomposition is exact (inputs.planted_exact).

Tolerances:
  * product: each operand vector is held as an integer of 2t - 2 = 322 bits
    relative to its largest entry (t = 162 for K <= 4096; as two halves of t
    bits), so each entry of the product is within K 2^-321 max|a_i| max|b_j| of
    the exact product of the given operands, and within 2^-318 of itself after
    its rounding to six words; the bound used is (K + 4) 2^-316 max|a_i| max|b_j|;
  * refined factors: exact residuals <= 1e-93 n (the stop test's tolerance);
    Q within 1e-90 of the exact Q0 and of the oracle's factor, up to column
    signs, and the diagonal of T^ within 1e-90 ||A||_F of the planted
    eigenvalues (gap 1/64).
"""
import numpy as np
import pytest

from oracle import mptarget as mp
from paper_2203_10879_gb300 import _binding as B
from paper_2203_10879_gb300 import inputs
from gpu_util import from_dev, to_dev

pytestmark = pytest.mark.gpu
F = mp.FBITS_D6
W = 6


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    B.lib()
    return torch


def _opts(**kw):
    base = dict(target=B.SR_TARGET_D6, lp=B.SR_LP_FP64, qhat_type=B.SR_QHAT_FP64, hp_gemm=B.SR_HP_OZAKI_CRT)
    base.update(kw)
    return B.default_options(**base)


def _handle(n_max, **kw):
    s, h = B.schur_refine_create(n_max, _opts(**kw), None)
    assert s == B.SR_OK, B.status_string(s)
    return h


def _dev(planes):
    return to_dev(np.hstack(planes))


def _host(t):
    a = from_dev(t)
    c = a.shape[1] // W
    return tuple(np.asfortranarray(a[:, k * c:(k + 1) * c]) for k in range(W))


def _empty(torch, n, c):
    return torch.zeros((W * c, n), dtype=torch.float64, device="cuda").t()


def _ulp(x):
    return np.abs(np.nextafter(x, np.inf) - x)


def test_d6_options_gate(torch):
    for kw in (dict(hp_gemm=B.SR_HP_FP64), dict(lp=B.SR_LP_FP32), dict(qhat_type=B.SR_QHAT_FP32), dict(graph=1)):
        s, h = B.schur_refine_create(64, _opts(**kw), None)
        assert s == B.SR_ERR_UNSUPPORTED and not h.value, kw
    s, h = B.schur_refine_create(64, _opts(ozaki_slices=16), None)
    assert s == B.SR_ERR_INVALID_ARG and not h.value


def _random(rng, rows, cols, spread=20):
    """Six planes with row scales 2^U(-spread, spread), each word about 2^-54
    of the one before."""
    sc = np.exp2(rng.integers(-spread, spread + 1, (rows, 1))).astype(float)
    p = [rng.standard_normal((rows, cols)) * sc]
    for _ in range(W - 1):
        p.append(p[-1] * rng.uniform(-1, 1, (rows, cols)) * 2.0 ** -54)
    return tuple(np.asfortranarray(x) for x in p)


@pytest.mark.parametrize("n,transA", [(64, 0), (100, 0), (129, 1)])
def test_d6_product_matches_exact_product(torch, n, transA):
    rng = np.random.default_rng(n + 5 * transA)
    A = _random(rng, n, n)
    Bm = tuple(np.asfortranarray(p.T) for p in _random(rng, n, n))   # columns with their own scales
    h = _handle(n)
    try:
        C = _empty(torch, n, n)
        s = B.schur_refine_gemm(h, transA, n, n, n, _dev(A), _dev(Bm), C)
        assert s == B.SR_OK, B.status_string(s)
        Cw = _host(C)
    finally:
        B.schur_refine_destroy(h)
    Af = mp.to_fx(A, F)
    Af = Af.T if transA else Af
    exact = np.dot(Af, mp.to_fx(Bm, F))                                 # scale 2^-2F
    got = mp.to_fx(Cw, F) * (1 << F)
    amax = np.abs(A[0].T if transA else A[0]).max(axis=1)
    bmax = np.abs(Bm[0]).max(axis=0)
    for i in range(n):
        for j in range(n):
            bound = (n + 4) * 2.0 ** -316 * amax[i] * bmax[j]
            assert abs(int(got[i, j]) - int(exact[i, j])) <= mp._f2i(bound, 2 * F), (i, j)
    for k in range(1, W):
        nz = Cw[k - 1] != 0
        assert np.all(np.abs(Cw[k][nz]) <= _ulp(Cw[k - 1][nz]) / 2)


def _refine(p, torch):
    n = p.n
    h = _handle(n)
    try:
        z = np.zeros_like(p.A)
        A = _dev((p.A,) + (z,) * (W - 1))
        Q = _empty(torch, n, n)
        T = _empty(torch, n, n)
        st, nr = B.schur_refine_step(h, n, A, Q, to_dev(p.Qhat), T)
        rs, rT, rQ = B.schur_refine_residuals(h, n, A, Q)
        assert rs == B.SR_OK
        return st, nr, _host(Q), _host(T), (rT, rQ)
    finally:
        B.schur_refine_destroy(h)


def _max_diff_words(Xw, Y):
    """max |(x0 + ... + x5) - Y| in float64: x0 - Y is exact and each later word
    nearly cancels what is left."""
    d = Xw[0] - Y
    for k in range(1, W):
        d = d + Xw[k]
    return np.max(np.abs(d))


@pytest.mark.parametrize("n", [32, 64])
def test_d6_refinement_matches_oracle(torch, n):
    p = inputs.unit_step_exact(n)
    st, nr, Qw, Tw, (rT, rQ) = _refine(p, torch)
    tol = mp.default_tol_d6(n)
    ref = mp.refine_fx(p.A, p.Qhat, tol=tol, F=F)
    assert ref.status == 0 and st == B.SR_OK, B.status_string(st)
    assert nr.iters == ref.iters == 7 and nr.hp_gemms == 4 * nr.iters
    cT, cQ = mp.residuals_exact(p.A, Qw, F=F)
    assert cT <= tol and cQ <= tol
    assert rT <= tol and rQ <= tol
    s = np.sign(np.sum(Qw[0] * p.Q0, axis=0))
    s[s == 0] = 1.0
    assert _max_diff_words(Qw, p.Q0 * s) <= 1e-90
    d = mp.to_fx(Qw, F) - mp.to_fx(mp.to_words(ref.Q, F, W), F)
    assert max(abs(int(v)) for v in d.ravel()) <= mp._f2i(1e-90, F)
    assert _max_diff_words(tuple(np.diag(t) for t in Tw), p.lam) <= 1e-90 * np.linalg.norm(p.A)


def test_d6_workload_size(torch):
    # the six-double workload (n = 1024, lambda_k = 1 + k/64): the refined factor
    # against the exact Q0 over every entry, the Schur diagonal against lambda
    p = inputs.unit_step_exact(1024)
    st, nr, Qw, Tw, (rT, rQ) = _refine(p, torch)
    assert st == B.SR_OK, B.status_string(st)
    assert nr.iters == 7
    tol = mp.default_tol_d6(1024)
    assert rT <= tol and rQ <= tol
    s = np.sign(np.sum(Qw[0] * p.Q0, axis=0))
    s[s == 0] = 1.0
    assert _max_diff_words(Qw, p.Q0 * s) <= 1e-90
    assert _max_diff_words(tuple(np.diag(t) for t in Tw), p.lam) <= 1e-90 * np.linalg.norm(p.A)
