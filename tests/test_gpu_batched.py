"""schur_refine_batched: many independent matrices of uneven order (the batched
workload: n log-uniform in [32, 512], each built like the unit-step problem).

Each matrix must meet the same bar as a single refinement (residuals certified
in double-double <= 1e-14 sqrt(n); Q columns against the oracle and the planted
Q0 up to sign within 1e-12, gaps 1/64 >= 1e-2), and the worker pool must give
bit-for-bit the results of the one-matrix-at-a-time loop (same kernels, same
data, integer-exact emulated products).
"""
import numpy as np
import pytest

import oracle
from paper_2203_10879_gb300 import _binding as B
from paper_2203_10879_gb300 import inputs
from gpu_util import from_dev, sign_align, to_dev

pytestmark = pytest.mark.gpu


def _run(problems, workers, **kw):
    import torch
    nmax = max(p.n for p in problems)
    s, h = B.schur_refine_create(nmax, B.default_options(batch_streams=workers, **kw), None)
    assert s == B.SR_OK
    try:
        As = [to_dev(p.A) for p in problems]
        Qh = [to_dev(p.Qhat) for p in problems]
        Qs = [torch.zeros((p.n, p.n), dtype=torch.float64, device="cuda").t() for p in problems]
        st, iters, stats = B.schur_refine_batched(h, [p.n for p in problems], As, Qs, Qh)
        torch.cuda.synchronize()
        return st, iters, stats, [from_dev(q) for q in Qs]
    finally:
        B.schur_refine_destroy(h)


@pytest.fixture(scope="module")
def batch():
    ns = inputs.batch_sizes(20)
    return [inputs.batch_problem(i, n) for i, n in enumerate(ns)]


@pytest.mark.parametrize("hp", [B.SR_HP_OZAKI_BF16, B.SR_HP_FP64])
def test_batched_matches_oracle(batch, hp):
    st, iters, stats, Qs = _run(batch, 4, hp_gemm=hp, lp=B.SR_LP_FP32)
    assert st == B.SR_OK and all(x == B.SR_OK for x in stats)
    for p, Q, k in zip(batch, Qs, iters):
        ref = oracle.refine(p.A, p.Qhat, lp="f32")
        assert ref.status == oracle.OK and abs(k - ref.iters) <= 1
        tol = oracle.default_tol(p.n)
        cT, cQ = oracle.residuals_dd(p.A, Q)
        assert cT <= tol and cQ <= tol, (p.n, cT, cQ)
        assert np.max(np.abs(sign_align(Q, ref.Q) - ref.Q)) <= 1e-12
        assert np.max(np.abs(sign_align(Q, p.Q0) - p.Q0)) <= 1e-12


def test_worker_pool_equals_serial_loop(batch):
    sub = batch[:8]
    _, it1, s1, Q1 = _run(sub, 1, hp_gemm=B.SR_HP_OZAKI_BF16)
    _, it4, s4, Q4 = _run(sub, 4, hp_gemm=B.SR_HP_OZAKI_BF16)
    assert it1 == it4 and s1 == s4
    for a, b in zip(Q1, Q4):
        assert np.array_equal(a, b)


def test_batched_rejects_bad_sizes():
    import torch
    s, h = B.schur_refine_create(64, B.default_options(), None)
    try:
        A = to_dev(np.eye(128))
        st, _, _ = B.schur_refine_batched(h, [128], [A], [A], None)
        assert st == B.SR_ERR_INVALID_ARG
        st, _, _ = B.schur_refine_batched(h, [], [], [], None)
        assert st == B.SR_OK
    finally:
        B.schur_refine_destroy(h)
