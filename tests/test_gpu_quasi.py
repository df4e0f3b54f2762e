"""GPU parity of the real quasi-triangular Schur form (Sec. 3, real Schur
decompositions: 2 x 2 diagonal blocks for complex-conjugate pairs), through
the C ABI, against the oracle.

Tolerances:
  * the block solve in FP64 agrees with the oracle's block Alg. 2 to a few
    hundred u64 relative to |L| on the well-separated test spectra (the sums
    run in another admissible order; each block equation is the same
    Kronecker system); in FP32 both are off the FP64 solution by O(u32 |L|),
    and the GPU's error is compared with the oracle's own FP32 error;
  * blocks that would straddle the solver's 32-row tiles (a 2 x 2 block
    starting on row 31 or 63) are included on purpose: the library pads them;
  * refined factors: the residual below the diagonal blocks and ||Q^T Q - I||
    certified in double-double by the oracle <= 1e-14 sqrt(n), the blocks read
    off the final T^ equal to the planted ones, and their eigenvalues within
    1e-12 of the planted complex pairs.
"""
import numpy as np
import pytest

import oracle
from paper_2203_10879_gb300 import _binding as B
from paper_2203_10879_gb300 import inputs
from gpu_util import from_dev, to_dev

pytestmark = pytest.mark.gpu
U64 = 2.0 ** -53
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available()
    B.lib()
    return torch


def _handle(n, **kw):
    s, h = B.schur_refine_create(n, B.default_options(quasi=1, **kw), None)
    assert s == B.SR_OK, B.status_string(s)
    return h


def _blocks(n, seed, force=(31, 63)):
    """Block array with random 2 x 2 blocks and blocks forced to start at the
    rows in `force` (the last rows of 32-row tiles)."""
    rng = np.random.default_rng(seed)
    blk = np.ones(n, dtype=np.int32)
    k = 0
    while k < n - 1:
        if k in force or (k + 1 not in force and rng.uniform() < 0.35):
            blk[k], blk[k + 1] = 2, 0
            k += 2
        else:
            k += 1
    return blk


def _problem(n, blk, seed):
    rng = np.random.default_rng(seed)
    mu = np.arange(n, dtype=float) / 4.0 + rng.uniform(0, 0.1, n)
    T = np.triu(rng.standard_normal((n, n)) * 0.05, 1)
    for k in range(n):
        if blk[k] == 2:
            a = 0.5 * (mu[k] + mu[k + 1])
            b = 0.1 + 0.1 * rng.uniform()
            T[k, k] = T[k + 1, k + 1] = a
            T[k, k + 1], T[k + 1, k] = 1.3 * b, -b / 1.3
        elif blk[k] == 1:
            T[k, k] = mu[k]
    E = np.where(oracle.block_lower_mask(blk), rng.standard_normal((n, n)) * 1e-3, 0.0)
    return T, E


SOLVE_MODES = [1, 2]   # the dataflow form (one launch), the stepwise form


def _gpu_solve(n, T, E, lp, solve_mode=0):
    dt = np.float32 if lp == B.SR_LP_FP32 else np.float64
    h = _handle(n, lp=lp, solve_mode=solve_mode)
    try:
        TE = to_dev((T + E).astype(dt))
        s = B.schur_refine_trisolve(h, n, TE, to_dev(np.diagonal(T).copy()))
        out = from_dev(TE)
    finally:
        B.schur_refine_destroy(h)
    return s, out


@pytest.mark.parametrize("solve_mode", SOLVE_MODES)
@pytest.mark.parametrize("n", [2, 5, 33, 64, 100, 257])
def test_quasi_trisolve_fp64_parity(torch, n, solve_mode):
    blk = _blocks(n, n)
    T, E = _problem(n, blk, 3 * n)
    s, out = _gpu_solve(n, T, E, B.SR_LP_FP64, solve_mode)
    assert s == B.SR_OK, B.status_string(s)
    mask = oracle.block_lower_mask(blk)
    L = np.where(mask, out, 0.0)
    assert np.array_equal(np.triu(out), np.triu(T))            # T (upper part) untouched
    assert np.all(out[np.tril(np.ones((n, n), bool), -1) & ~mask] == 0)   # couplings cleared
    ref = oracle.alg2_quasi(T, E, blk, np.diagonal(T).copy())
    scale = max(np.max(np.abs(ref)), 1e-300)
    assert np.max(np.abs(L - ref)) <= 1e3 * U64 * scale


@pytest.mark.parametrize("solve_mode", SOLVE_MODES)
@pytest.mark.parametrize("n", [33, 100, 257, 700, 1500])
def test_quasi_trisolve_fp32_parity(torch, n, solve_mode):
    blk = _blocks(n, n + 1)
    T, E = _problem(n, blk, 5 * n)
    s, out = _gpu_solve(n, T, E, B.SR_LP_FP32, solve_mode)
    assert s == B.SR_OK, B.status_string(s)
    mask = oracle.block_lower_mask(blk)
    L32 = np.where(mask, out.astype(np.float64), 0.0)
    d = np.diagonal(T).copy()
    L64 = oracle.alg2_quasi(T, E, blk, d)
    Lo32 = oracle.alg2_quasi(T.astype(np.float32), E.astype(np.float32), blk, d).astype(np.float64)
    e_gpu = np.linalg.norm(L32 - L64)
    e_orc = np.linalg.norm(Lo32 - L64)
    assert e_gpu <= 20 * max(e_orc, U32 * np.linalg.norm(L64))


@pytest.mark.parametrize("solve_mode", SOLVE_MODES)
def test_quasi_trisolve_shared_pair_is_nondistinct(torch, solve_mode):
    n = 40
    blk = np.ones(n, dtype=np.int32)
    for k in (4, 20):
        blk[k], blk[k + 1] = 2, 0
    T, E = _problem(n, blk, 9)
    T[20:22, 20:22] = T[4:6, 4:6]           # the same complex pair twice
    s, _ = _gpu_solve(n, T, E, B.SR_LP_FP64, solve_mode)
    assert s == B.SR_ERR_NONDISTINCT


def _refine(p, hp, **kw):
    import torch
    n = p.n
    h = _handle(n, hp_gemm=hp, lp=B.SR_LP_FP32, **kw)
    try:
        A = to_dev(p.A)
        Q = torch.zeros((n, n), dtype=torch.float64, device="cuda").t()
        T = torch.zeros((n, n), dtype=torch.float64, device="cuda").t()
        st, nr = B.schur_refine_step(h, n, A, Q, to_dev(p.Qhat), T)
        rs, rT, rQ = B.schur_refine_residuals(h, n, A, Q)
        assert rs == B.SR_OK
        return st, nr, from_dev(Q), from_dev(T), (rT, rQ)
    finally:
        B.schur_refine_destroy(h)


@pytest.mark.parametrize("hp,solve_mode", [(B.SR_HP_OZAKI_CRT, 1), (B.SR_HP_OZAKI_CRT, 2), (B.SR_HP_FP64, 0)])
@pytest.mark.parametrize("n", [64, 300])
def test_quasi_refinement_matches_oracle(torch, n, hp, solve_mode):
    p = inputs.quasi_real(n)
    st, nr, Q, T, (rT, rQ) = _refine(p, hp, solve_mode=solve_mode)
    ref = oracle.refine(p.A, p.Qhat, lp="f32", quasi=True)
    assert ref.status == oracle.OK
    assert st == B.SR_OK, B.status_string(st)
    assert abs(nr.iters - ref.iters) <= 1 and nr.hp_gemms == 4 * nr.iters
    blk = oracle.quasi_blocks(T)
    assert np.array_equal(blk, p.blk)
    tol = oracle.default_tol(n)
    cT, cQ = oracle.residuals_dd(p.A, Q, blk=blk)
    assert cT <= tol and cQ <= tol
    # the library's own double-double residuals of a quasi handle skip the couplings too
    assert rT == pytest.approx(cT, rel=1e-6, abs=1e-30) and rQ == pytest.approx(cQ, rel=1e-6, abs=1e-30)
    ev = np.zeros(n, dtype=np.complex128)
    for k in range(n):
        if blk[k] == 2:
            w = np.linalg.eigvals(T[k:k + 2, k:k + 2])
            ev[k], ev[k + 1] = w[np.argmax(w.imag)], w[np.argmin(w.imag)]
        elif blk[k] == 1:
            ev[k] = T[k, k]
    assert np.max(np.abs(ev - p.lam)) <= 1e-12


def test_quasi_solve_forms_agree(torch):
    # both launch forms solve the same block equations on a ragged order of many
    # tiles: they agree to the working precision's rounding
    n = 1000
    blk = _blocks(n, 17)
    T, E = _problem(n, blk, 19)
    outs = []
    for mode in SOLVE_MODES:
        s, out = _gpu_solve(n, T, E, B.SR_LP_FP32, mode)
        assert s == B.SR_OK
        outs.append(np.where(oracle.block_lower_mask(blk), out.astype(np.float64), 0.0))
    assert np.linalg.norm(outs[0] - outs[1]) <= 100 * U32 * np.linalg.norm(outs[1])


def test_quasi_workload_n1000(torch):
    p = inputs.quasi_real(1000)
    st, nr, Q, T, (rT, rQ) = _refine(p, B.SR_HP_OZAKI_CRT)
    assert st == B.SR_OK, B.status_string(st)
    tol = oracle.default_tol(1000)
    blk = oracle.quasi_blocks(T)
    assert np.array_equal(blk, p.blk)
    cT, cQ = oracle.residuals_dd(p.A, Q, blk=blk)
    assert cT <= tol and cQ <= tol


def test_triangular_form_fails_on_complex_pairs(torch):
    # the same input through the triangular form: a real T cannot hold a complex
    # pair on its diagonal, and the iteration breaks down (as the oracle's does)
    p = inputs.quasi_real(64)
    s, h = B.schur_refine_create(64, B.default_options(hp_gemm=B.SR_HP_OZAKI_CRT, lp=B.SR_LP_FP32), None)
    assert s == B.SR_OK
    try:
        import torch as _t
        Q = _t.zeros((64, 64), dtype=_t.float64, device="cuda").t()
        st, _ = B.schur_refine_step(h, 64, to_dev(p.A), Q, to_dev(p.Qhat))
    finally:
        B.schur_refine_destroy(h)
    ref = oracle.refine(p.A, p.Qhat, lp="f32")
    assert st != B.SR_OK and ref.status != oracle.OK


def test_quasi_option_gate(torch):
    for kw in ({"dtype": B.SR_COMPLEX, "hp_gemm": B.SR_HP_OZAKI_CRT}, {"graph": 1}, {"symmetric": 1}):
        s, h = B.schur_refine_create(64, B.default_options(quasi=1, **kw), None)
        assert s == B.SR_ERR_UNSUPPORTED and not h.value
