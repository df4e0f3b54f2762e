"""GPU parity of the emulated FP64 products (bf16 digits on tcgen05) and of the
refinement that uses them.

Tolerances:
  * integer-valued operands with |entries| < 2^7 are split exactly into one
    digit each, every product is an exact integer, so the result is bit-exact;
  * with s digits each scaled operand x = a 2^-e in (-1, 1) is held in fixed
    point to 2^-(7+8(s-1)+1), and the dropped digit pairs (p+q >= s, at most s
    per level, each <= 2^14 2^(-14-8(p+q))) weigh at most ~s 2^(-8s); so per
    term |ab - emulated| <= (s+2) 2^(-8s) 2^(e_i+f_j) and over k terms
    |C - AB| <= k (s+3) 2^(-8s) 2^(e_i+f_j) entrywise. For s = 7 this is the
    size of the FP64 bound k u |A||B|, against which the products are checked
    (reference: the oracle's double-double product).
"""
import numpy as np
import pytest

import oracle
from paper_2203_10879_gb300 import _binding as B
from paper_2203_10879_gb300 import inputs
from gpu_util import from_dev, sign_align, to_dev

pytestmark = pytest.mark.gpu
U64 = 2.0 ** -53


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available()
    return torch


def _gemm(torch, A, Bm, transA, slices=0):
    m = A.shape[1] if transA else A.shape[0]
    k = A.shape[0] if transA else A.shape[1]
    n = Bm.shape[1]
    s, h = B.schur_refine_create(max(m, n, k), B.default_options(hp_gemm=B.SR_HP_OZAKI_BF16, ozaki_slices=slices),
                                 None)
    assert s == B.SR_OK, B.status_string(s)
    try:
        C = torch.zeros((n, m), dtype=torch.float64, device="cuda").t()
        st = B.schur_refine_gemm(h, int(transA), m, n, k, to_dev(A), to_dev(Bm), C)
        assert st == B.SR_OK, B.status_string(st)
        return from_dev(C)
    finally:
        B.schur_refine_destroy(h)


def test_ozaki_single_tile_exact_integers(torch):
    rng = np.random.default_rng(1)
    A = rng.integers(-100, 101, (128, 256)).astype(np.float64)
    Bm = rng.integers(-100, 101, (256, 128)).astype(np.float64)
    C = _gemm(torch, A, Bm, False)
    assert np.array_equal(C, A @ Bm)


@pytest.mark.parametrize("m,n,k,transA", [(200, 130, 300, False), (129, 257, 513, True), (1, 3, 2, False)])
def test_ozaki_exact_integers_ragged(torch, m, n, k, transA):
    rng = np.random.default_rng(m + n + k)
    A = rng.integers(-127, 128, (k, m) if transA else (m, k)).astype(np.float64)
    Bm = rng.integers(-127, 128, (k, n)).astype(np.float64)
    C = _gemm(torch, A, Bm, transA)
    opA = A.T if transA else A
    assert np.array_equal(C, opA @ Bm)


@pytest.mark.parametrize("m,n,k,transA", [(160, 96, 700, True), (300, 300, 300, False)])
def test_ozaki_fp64_accuracy_vs_double_double(torch, m, n, k, transA):
    rng = np.random.default_rng(7 * m + k)
    A = rng.standard_normal((k, m) if transA else (m, k)) * np.exp(rng.uniform(-3, 3, (1, m) if transA else (m, 1)))
    Bm = rng.standard_normal((k, n))
    C = _gemm(torch, A, Bm, transA)
    hi, lo = oracle.gemm_dd(A, None, Bm, None, transA=transA)
    opA = A.T if transA else A
    err = np.abs(C - hi - lo)
    bound = k * U64 * (np.abs(opA) @ np.abs(Bm))
    assert np.all(err <= bound)
    # and clearly better than the bound on average (the split error is ~2^-55 per term)
    assert np.median(err / bound) < 0.1


@pytest.mark.parametrize("s", [2, 3, 5])
def test_ozaki_digit_count_error_law(torch, s):
    rng = np.random.default_rng(s)
    m = n = k = 256
    A = rng.standard_normal((m, k))
    Bm = rng.standard_normal((k, n))
    C = _gemm(torch, A, Bm, False, slices=s)
    hi, lo = oracle.gemm_dd(A, None, Bm, None)
    ea = np.ceil(np.log2(np.max(np.abs(A), axis=1) * (1 + 2 ** -52)))
    fb = np.ceil(np.log2(np.max(np.abs(Bm), axis=0) * (1 + 2 ** -52)))
    scale = 2.0 ** (ea[:, None] + fb[None, :])
    bound = k * (s + 3) * 2.0 ** (-8 * s) * scale
    err = np.abs(C - hi - lo)
    assert np.all(err <= bound)
    assert np.max(err / bound) > 1e-4   # s digits really truncate: not secretly exact


def test_ozaki_nonfinite_input_gives_nan(torch):
    A = np.ones((64, 64))
    A[5, 7] = np.inf
    C = _gemm(torch, A, np.ones((64, 64)), False)
    assert np.all(np.isnan(C[5, :]))
    assert np.all(np.isfinite(np.delete(C, 5, axis=0)))


def _refine(p, **kw):
    import torch
    n = p.n
    s, h = B.schur_refine_create(n, B.default_options(hp_gemm=B.SR_HP_OZAKI_BF16, **kw), None)
    assert s == B.SR_OK
    try:
        A, Qhat = to_dev(p.A), to_dev(p.Qhat)
        Q = torch.zeros((n, n), dtype=torch.float64, device="cuda").t()
        st, nr = B.schur_refine_step(h, n, A, Q, Qhat)
        return st, nr, from_dev(Q)
    finally:
        B.schur_refine_destroy(h)


def test_refine_ozaki_unit_step_n64(torch):
    p = inputs.unit_step_real(64)
    st, nr, Q = _refine(p, lp=B.SR_LP_FP32)
    ref = oracle.refine(p.A, p.Qhat, lp="f32")
    assert st == B.SR_OK and nr.iters == ref.iters
    tol = oracle.default_tol(64)
    cT, cQ = oracle.residuals_dd(p.A, Q)
    assert cT <= tol and cQ <= tol
    assert np.max(np.abs(sign_align(Q, ref.Q) - ref.Q)) <= 1e-12
    assert np.max(np.abs(sign_align(Q, p.Q0) - p.Q0)) <= 1e-12


@pytest.mark.parametrize("n", [300, 1000])
def test_refine_ozaki_jittered(torch, n):
    p = inputs.jittered_real(n)
    st, nr, Q = _refine(p, lp=B.SR_LP_FP32)
    ref = oracle.refine(p.A, p.Qhat, lp="f32")
    assert st == B.SR_OK and abs(nr.iters - ref.iters) <= 1
    tol = oracle.default_tol(n)
    cT, cQ = oracle.residuals_dd(p.A, Q)
    assert cT <= tol and cQ <= tol
    Tq = np.diagonal(Q.T @ p.A @ Q)
    Tr = np.diagonal(ref.Q.T @ p.A @ ref.Q)
    assert np.max(np.abs(Tq - Tr)) <= 1e-12


def test_one_pass_parity_ozaki(torch):
    # one pass through the emulated engine against the oracle's FP32 pass: the
    # FP32 solve dominates the difference, O(u32 ||W||) in Q
    p = inputs.planted(96, inputs.eig_unit_step(96), 5, pert=1e-5)
    st, nr, Q = _refine(p, lp=B.SR_LP_FP32, max_iter=1)
    assert st == B.SR_ERR_NOT_CONVERGED and nr.iters == 1
    Q0, _ = oracle.ns_init(p.Qhat)
    Q1, info = oracle.iteration(p.A, Q0, lp="f32")
    assert nr.w_norm == pytest.approx(info.w_norm, rel=1e-5)
    assert np.max(np.abs(Q - Q1)) <= 50 * 2.0 ** -24 * info.w_norm + 1e-13


def test_refine_ozaki_full_sigma(torch):
    p = inputs.jittered_real(257)
    st, nr, Q = _refine(p, lp=B.SR_LP_FP32, full_sigma=1)
    ref = oracle.refine(p.A, p.Qhat, lp="f32", full_sigma=True)
    assert st == B.SR_OK and abs(nr.iters - ref.iters) <= 1
    tol = oracle.default_tol(257)
    cT, cQ = oracle.residuals_dd(p.A, Q)
    assert cT <= tol and cQ <= tol
    assert np.max(np.abs(sign_align(Q, ref.Q) - ref.Q)) <= 1e-9


def test_autotuned_work_split_gives_identical_results(torch):
    # the level groups of the slice products write disjoint exact integer planes:
    # whichever split the autotuner keeps, the refinement is bit-for-bit the same
    p = inputs.jittered_real(1000)
    out = []
    for tune in (0, 1):
        st, h = B.schur_refine_create(1000, B.default_options(hp_gemm=B.SR_HP_OZAKI_BF16, lp=B.SR_LP_FP32,
                                                              tune=tune), None)
        assert st == B.SR_OK
        try:
            Q = torch.zeros((1000, 1000), dtype=torch.float64, device="cuda").t()
            s, nr = B.schur_refine_step(h, 1000, to_dev(p.A), Q, to_dev(p.Qhat))
            s2, nr2 = B.schur_refine_step(h, 1000, to_dev(p.A), Q, to_dev(p.Qhat))   # tuned shapes reused
            assert s == s2 == B.SR_OK and nr.iters == nr2.iters
            out.append(from_dev(Q))
        finally:
            B.schur_refine_destroy(h)
    assert np.array_equal(out[0], out[1])
