"""GPU parity of the double-double target (hp = double-double, lp = FP64).

The CUDA library, called through its C ABI, against the double-double oracle
(``oracle.ddtarget``) on the planted double-double workload. Tolerances:
  * a double-double product of depth k is within about k 2^-104 |A||B| of the
    exact one (oracle: triple loop with TwoProd/TwoSum); the emulated product
    with 14 bf16 digits per operand drops terms below (s + 2) 2^-8s of the
    vector scales, about k 2^-108 max|a_i| max|b_j|; the bound used is
    8 k 2^-104 times the row and column maxima;
  * the residue form (32 moduli) holds every operand as an integer of t bits
    (t = 113 to 115 at these inner lengths), so its product is within
    k 2^-t of the row and column maxima: inside the same bound;
  * integer operands make every product exact: bit-exact agreement;
  * the FP64 solve with double-double divisors agrees with the oracle's Alg. 2
    to a few hundred u64 relative to |L|;
  * refined factors: residuals <= 1e-28 n (double-double on the device, 128-bit
    floating point in the oracle), columns of Q within 1e-25 of the oracle's
    and of the planted Q0 up to sign (eigenvalue gap 1/64).
"""
import numpy as np
import pytest

import oracle
from oracle import ddtarget as D
from paper_2203_10879_gb300 import _binding as B
from paper_2203_10879_gb300 import inputs
from gpu_util import from_dev, to_dev

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53
U_DD = 2.0 ** -104
ENGINES = [B.SR_HP_OZAKI_BF16, B.SR_HP_OZAKI_CRT, B.SR_HP_FP64]
EMULATED = [B.SR_HP_OZAKI_BF16, B.SR_HP_OZAKI_CRT]


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    B.lib()
    return torch


def _handle(n_max, hp, **kw):
    o = B.default_options(target=B.SR_TARGET_DD, lp=B.SR_LP_FP64, qhat_type=B.SR_QHAT_FP64, hp_gemm=hp, **kw)
    s, h = B.schur_refine_create(n_max, o, None)
    assert s == B.SR_OK, B.status_string(s)
    return h


def _dd_dev(hi, lo):
    return to_dev(np.hstack([hi, lo]))


def _dd_host(t):
    a = from_dev(t)
    c = a.shape[1] // 2
    return a[:, :c], a[:, c:]


def _dd_empty(torch, n, c):
    return torch.zeros((2 * c, n), dtype=torch.float64, device="cuda").t()


def _dd_random(rng, shape):
    hi = rng.standard_normal(shape)
    lo = hi * rng.uniform(-1, 1, shape) * 2.0 ** -53
    return hi, (hi + lo) - hi


def test_dd_options_gate(torch):
    bad = [dict(target=B.SR_TARGET_DD),                                           # FP32 lp
           dict(target=B.SR_TARGET_DD, lp=B.SR_LP_FP64),                          # FP32 Qhat
           dict(target=B.SR_TARGET_DD, lp=B.SR_LP_FP64, qhat_type=B.SR_QHAT_FP64, dtype=B.SR_COMPLEX,
                hp_gemm=B.SR_HP_OZAKI_BF16)]
    for kw in bad:
        s, h = B.schur_refine_create(64, B.default_options(**kw), None)
        assert s == B.SR_ERR_UNSUPPORTED and not h.value
    s, h = B.schur_refine_create(64, B.default_options(target=B.SR_TARGET_DD, lp=B.SR_LP_FP64,
                                                       qhat_type=B.SR_QHAT_FP64, ozaki_slices=15), None)
    assert s == B.SR_ERR_INVALID_ARG


@pytest.mark.parametrize("hp", ENGINES)
@pytest.mark.parametrize("m,n,k,transA", [(100, 77, 129, 0), (257, 33, 300, 1), (1, 5, 3, 0), (300, 260, 520, 1)])
def test_dd_gemm_parity(torch, hp, m, n, k, transA):
    rng = np.random.default_rng(m + 7 * n + 13 * k + transA)
    A = _dd_random(rng, (k, m) if transA else (m, k))
    Bm = _dd_random(rng, (k, n))
    h = _handle(max(m, n, k), hp)
    try:
        C = _dd_empty(torch, m, n)
        s = B.schur_refine_gemm(h, transA, m, n, k, _dd_dev(*A), _dd_dev(*Bm), C)
        assert s == B.SR_OK, B.status_string(s)
        ch, cl = _dd_host(C)
        rh, rl = D.gemm(A, Bm, transA=bool(transA))
        diff = (ch - rh) + (cl - rl)
        opA = A[0].T if transA else A[0]
        bound = 8 * k * U_DD * np.outer(np.max(np.abs(opA), axis=1), np.max(np.abs(Bm[0]), axis=0))
        assert np.all(np.abs(diff) <= bound)
        assert np.max(np.abs(cl)) > 0          # the low planes carry information
    finally:
        B.schur_refine_destroy(h)


@pytest.mark.parametrize("hp", ENGINES)
def test_dd_gemm_exact_on_integers(torch, hp):
    rng = np.random.default_rng(3)
    m, n, k = 130, 200, 300
    A = (rng.integers(-1000, 1000, (m, k)).astype(float), np.zeros((m, k)))
    Bm = (rng.integers(-1000, 1000, (k, n)).astype(float), np.zeros((k, n)))
    h = _handle(max(m, n, k), hp)
    try:
        C = _dd_empty(torch, m, n)
        assert B.schur_refine_gemm(h, 0, m, n, k, _dd_dev(*A), _dd_dev(*Bm), C) == B.SR_OK
        ch, cl = _dd_host(C)
        assert np.array_equal(ch, A[0] @ Bm[0]) and np.all(cl == 0)
    finally:
        B.schur_refine_destroy(h)


@pytest.mark.parametrize("solve_mode", [1, 2])
@pytest.mark.parametrize("n", [2, 33, 100, 257, 500])
def test_dd_trisolve_parity(torch, n, solve_mode):
    rng = np.random.default_rng(n)
    d = 1.0 + np.arange(n) / 64.0
    dlo = rng.uniform(-1, 1, n) * 2.0 ** -54 * d
    dlo = (d + dlo) - d
    T = np.triu(rng.standard_normal((n, n)) / n, 1) + np.diag(d)
    E = np.tril(rng.standard_normal((n, n)) * 1e-14, -1)
    h = _handle(n, B.SR_HP_OZAKI_BF16, solve_mode=solve_mode)
    try:
        TE = to_dev(np.triu(T) + E)
        s = B.schur_refine_trisolve(h, n, TE, to_dev(np.concatenate([d, dlo])))
        assert s == B.SR_OK
        out = from_dev(TE)
        assert np.array_equal(np.triu(out), np.triu(T))
        ref = D.alg2_dd_divisors(T, E, (d, dlo))
        scale = max(np.max(np.abs(ref)), 1e-300)
        assert np.max(np.abs(np.tril(out, -1) - ref)) <= 1e3 * U64 * scale
    finally:
        B.schur_refine_destroy(h)


def test_dd_trisolve_low_parts_decide_divisor(torch):
    # equal FP64 diagonal entries, different low parts: divisor 2^-59 (not zero)
    T = np.array([[1.0, 0.25], [0.0, 1.0]])
    E = np.array([[0.0, 0.0], [3.0 * 2.0 ** -70, 0.0]])
    h = _handle(2, B.SR_HP_FP64)
    try:
        TE = to_dev(np.triu(T) + E)
        s = B.schur_refine_trisolve(h, 2, TE, to_dev(np.array([1.0, 1.0, -(2.0 ** -60), 2.0 ** -60])))
        assert s == B.SR_OK
        assert from_dev(TE)[1, 0] == -3.0 * 2.0 ** -70 / 2.0 ** -59
        TE = to_dev(np.triu(T) + E)
        assert B.schur_refine_trisolve(h, 2, TE, to_dev(np.array([1.0, 1.0, 0.0, 0.0]))) == B.SR_ERR_NONDISTINCT
    finally:
        B.schur_refine_destroy(h)


def _refine_gpu(torch, p, hp, **kw):
    n = p.n
    h = _handle(n, hp, **kw)
    try:
        A = _dd_dev(p.A_hi, p.A_lo)
        Q = _dd_empty(torch, n, n)
        T = _dd_empty(torch, n, n)
        s, nr = B.schur_refine_step(h, n, A, Q, to_dev(p.Qhat), T)
        rs, rT, rQ = B.schur_refine_residuals(h, n, A, Q)
        assert rs == B.SR_OK
        return s, nr, _dd_host(Q), _dd_host(T), (rT, rQ)
    finally:
        B.schur_refine_destroy(h)


@pytest.mark.parametrize("hp", ENGINES)
@pytest.mark.parametrize("n", [64, 100, 300])
def test_dd_refine_matches_oracle(torch, hp, n):
    p = inputs.unit_step_dd(n)
    s, nr, Q, T, (rT, rQ) = _refine_gpu(torch, p, hp)
    ref = D.refine_dd((p.A_hi, p.A_lo), p.Qhat)
    tol = D.default_tol_dd(n)
    assert s == B.SR_OK and ref.status == oracle.OK
    assert nr.iters == ref.iters and nr.hp_gemms == ref.hp_gemms == 4 * nr.iters
    assert rT <= tol and rQ <= tol, (rT, rQ, tol)
    oT, oQ = D.residuals_q((p.A_hi, p.A_lo), Q)
    assert oT <= tol and oQ <= tol, (oT, oQ, tol)
    sg = np.sign(np.sum(Q[0] * ref.Q[0], axis=0))
    dq = (Q[0] * sg - ref.Q[0]) + (Q[1] * sg - ref.Q[1])
    assert np.max(np.abs(dq)) <= 1e-25
    sg0 = np.sign(np.sum(Q[0] * p.Q0_hi, axis=0))
    dq0 = (Q[0] * sg0 - p.Q0_hi) + (Q[1] * sg0 - p.Q0_lo)
    assert np.max(np.abs(dq0)) <= 1e-25
    dlam = (np.diagonal(T[0]) - p.lam) + np.diagonal(T[1])
    assert np.max(np.abs(dlam)) <= 1e-26


def test_dd_engines_agree_and_full_sigma(torch):
    p = inputs.unit_step_dd(96)
    _, _, Qa, _, _ = _refine_gpu(torch, p, B.SR_HP_OZAKI_BF16)
    _, _, Qb, _, _ = _refine_gpu(torch, p, B.SR_HP_FP64)
    _, _, Qd, _, _ = _refine_gpu(torch, p, B.SR_HP_OZAKI_CRT)
    s, nr, Qc, _, (rT, rQ) = _refine_gpu(torch, p, B.SR_HP_OZAKI_BF16, full_sigma=1)
    assert s == B.SR_OK and rT <= D.default_tol_dd(96) and rQ <= D.default_tol_dd(96)
    for X in (Qb, Qc, Qd):
        assert np.max(np.abs((Qa[0] - X[0]) + (Qa[1] - X[1]))) <= 1e-26


@pytest.mark.parametrize("hp", EMULATED)
def test_dd_workload_full_size(torch, hp):
    """The n = 2048 double-double workload as the benchmark runs it: certified
    on the device, and sampled entries of Q^T A Q and Q^T Q - I of the GPU's Q
    evaluated by the oracle in 128-bit arithmetic."""
    n = 2048
    p = inputs.unit_step_dd(n)
    s, nr, Q, T, (rT, rQ) = _refine_gpu(torch, p, hp)
    tol = D.default_tol_dd(n)
    assert s == B.SR_OK and nr.iters <= 3
    assert rT <= tol and rQ <= tol, (rT, rQ, tol)
    rng = np.random.default_rng(2048)
    cols = rng.choice(n, 6, replace=False)
    rows = np.concatenate([rng.choice(n, 5, replace=False) for _ in cols] + [cols])
    cc = np.concatenate([np.repeat(cols, 5), cols])
    t, y = D.sample_entries_q((p.A_hi, p.A_lo), Q, rows, cc)
    anorm = np.linalg.norm(p.A_hi)
    for k, (i, j) in enumerate(zip(rows, cc)):
        tv = t[0][k] + t[1][k]
        if i > j:
            assert abs(tv) <= tol * anorm
        else:   # T^ from the device against the oracle's entry
            gv = (T[0][i, j] - t[0][k]) + (T[1][i, j] - t[1][k])
            assert abs(gv) <= 1e-28 * anorm
        assert abs(y[0][k] + y[1][k]) <= tol
    dlam = (np.diagonal(T[0]) - p.lam) + np.diagonal(T[1])
    assert np.max(np.abs(dlam)) <= 1e-25
