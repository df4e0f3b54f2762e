"""schur_refine_batched: many independent matrices of uneven order (the batched
workload: n log-uniform in [32, 512], each built like the unit-step problem).

Each matrix must meet the same bar as a single refinement (residuals certified
in double-double <= 1e-14 sqrt(n); Q columns against the oracle and the planted
Q0 up to sign within 1e-12, gaps 1/64 >= 1e-2). The grouped launches and the
worker pool must both give bit-for-bit the results of schur_refine_step on
each matrix alone (same kernels, same data, integer-exact emulated products,
the same tiles of the solve), and a matrix that fails must not disturb the
others.
"""
import numpy as np
import pytest

import oracle
from paper_2203_10879_gb300 import _binding as B
from paper_2203_10879_gb300 import inputs
from gpu_util import from_dev, sign_align, to_dev

pytestmark = pytest.mark.gpu


def _run(problems, workers, mode=0, **kw):
    import torch
    nmax = max(p.n for p in problems)
    s, h = B.schur_refine_create(nmax, B.default_options(batch_streams=workers, batch_mode=mode, **kw), None)
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


@pytest.mark.parametrize("hp", [B.SR_HP_OZAKI_BF16, B.SR_HP_OZAKI_CRT, B.SR_HP_FP64])
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
    _, it1, s1, Q1 = _run(sub, 1, mode=1, hp_gemm=B.SR_HP_OZAKI_BF16)
    _, it4, s4, Q4 = _run(sub, 4, mode=1, hp_gemm=B.SR_HP_OZAKI_BF16)
    assert it1 == it4 and s1 == s4
    for a, b in zip(Q1, Q4):
        assert np.array_equal(a, b)


def _single(p, **kw):
    import torch
    s, h = B.schur_refine_create(p.n, B.default_options(**kw), None)
    assert s == B.SR_OK
    try:
        Q = torch.zeros((p.n, p.n), dtype=torch.float64, device="cuda").t()
        st, nr = B.schur_refine_step(h, p.n, to_dev(p.A), Q, to_dev(p.Qhat))
        return st, nr.iters, from_dev(Q)
    finally:
        B.schur_refine_destroy(h)


@pytest.mark.parametrize("hp", [B.SR_HP_OZAKI_BF16, B.SR_HP_OZAKI_CRT])
@pytest.mark.parametrize("solve_mode", [1, 2])
def test_grouped_launches_equal_single_steps(batch, solve_mode, hp):
    # the residue form: each matrix's residues, products and rebuild use the
    # fixed-point bits t of its own order, as a single step on it does
    st, iters, stats, Qs = _run(batch, 8, mode=0, hp_gemm=hp, solve_mode=solve_mode)
    assert st == B.SR_OK
    for p, Q, k, s in zip(batch, Qs, iters, stats):
        s1, k1, Q1 = _single(p, hp_gemm=hp, solve_mode=solve_mode)
        assert (s, k) == (s1, k1), p.n
        if solve_mode == 2:
            assert np.array_equal(Q, Q1), p.n
        else:
            # a single matrix's dataflow solve hands its far products to helper
            # tasks (another FP32 summation order than the group form's): the
            # refined factors agree to FP64 rounding
            assert np.max(np.abs(Q - Q1)) <= 1e-13, p.n


@pytest.mark.parametrize("hp", [B.SR_HP_OZAKI_BF16, B.SR_HP_OZAKI_CRT])
def test_grouped_launches_isolate_a_failing_matrix(batch, hp):
    # the variance reading of the upper entries (std 1/sqrt(n)) on a packed
    # spectrum diverges (the analogue of Example 3); its neighbours must not care
    bad = inputs.jittered_real(200, upper_std=1.0 / np.sqrt(200))
    group = batch[:5] + [bad] + batch[5:9]
    st, iters, stats, Qs = _run(group, 8, mode=0, hp_gemm=hp)
    assert stats[5] in (B.SR_ERR_NONFINITE, B.SR_ERR_NOT_CONVERGED, B.SR_ERR_NONDISTINCT)
    assert st == stats[5]
    _, _, _, Qok = _run(batch[:9], 8, mode=0, hp_gemm=hp)
    for a, b, s in zip(Qs[:5] + Qs[6:], Qok, stats[:5] + stats[6:]):
        assert s == B.SR_OK
        assert np.array_equal(a, b)


def test_grouped_launches_grow_and_reuse_workspace(batch):
    import torch
    nmax = max(p.n for p in batch)
    s, h = B.schur_refine_create(nmax, B.default_options(hp_gemm=B.SR_HP_OZAKI_BF16), None)
    assert s == B.SR_OK
    try:
        for group in (batch[:3], batch, batch[2:6]):
            As = [to_dev(p.A) for p in group]
            Qh = [to_dev(p.Qhat) for p in group]
            Qs = [torch.zeros((p.n, p.n), dtype=torch.float64, device="cuda").t() for p in group]
            st, _, _ = B.schur_refine_batched(h, [p.n for p in group], As, Qs, Qh)
            assert st == B.SR_OK
            for p, Q in zip(group, Qs):
                tol = oracle.default_tol(p.n)
                cT, cQ = oracle.residuals_dd(p.A, from_dev(Q))
                assert cT <= tol and cQ <= tol
    finally:
        B.schur_refine_destroy(h)


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


@pytest.mark.parametrize("hp", [B.SR_HP_OZAKI_BF16, B.SR_HP_OZAKI_CRT])
def test_full_batched_workload_certified(hp):
    """The benchmarked group itself: all 1024 matrices of the batched workload in
    one schur_refine_batched call with the bench's options (both product forms). Every matrix's
    residuals are certified in double-double on the device
    (schur_refine_residuals, <= 1e-14 sqrt(n)); that certifier is checked against
    the oracle's double-double residuals on 25 matrices, the largest among them."""
    import torch
    ns = [int(n) for n in inputs.batch_sizes(1024)]
    nmax = max(ns)
    s, h = B.schur_refine_create(nmax, B.default_options(hp_gemm=hp, lp=B.SR_LP_FP32, batch_streams=8), None)
    assert s == B.SR_OK
    try:
        problems = [inputs.batch_problem(i, n) for i, n in enumerate(ns)]
        As = [to_dev(p.A) for p in problems]
        Qh = [to_dev(p.Qhat) for p in problems]
        Qs = [torch.zeros((n, n), dtype=torch.float64, device="cuda").t() for n in ns]
        st, iters, stats = B.schur_refine_batched(h, ns, As, Qs, Qh)
        torch.cuda.synchronize()
        assert st == B.SR_OK and all(x == B.SR_OK for x in stats)
        assert all(2 <= k <= 4 for k in iters)
        lib = []
        for n, A, Q in zip(ns, As, Qs):
            rs, rT, rQ = B.schur_refine_residuals(h, n, A, Q)
            assert rs == B.SR_OK
            tol = oracle.default_tol(n)
            assert rT <= tol and rQ <= tol, (n, rT, rQ)
            lib.append((rT, rQ))
        order = np.argsort(ns)
        sample = sorted(set(order[-4:].tolist() + list(range(0, 1024, 51))))
        for i in sample:
            cT, cQ = oracle.residuals_dd(problems[i].A, from_dev(Qs[i]))
            assert cT <= oracle.default_tol(ns[i]) and cQ <= oracle.default_tol(ns[i])
            assert lib[i][0] == pytest.approx(cT, rel=1e-6) and lib[i][1] == pytest.approx(cQ, rel=1e-6)
    finally:
        B.schur_refine_destroy(h)
