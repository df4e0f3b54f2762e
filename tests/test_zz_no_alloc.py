"""schur_refine_residuals_noalloc: the handle-free residual entry point.

It exists for callers that cannot call cudaMalloc (their device memory is owned
by a pool allocator, or allocation is forbidden after start-up); its scratch is
a fixed array in the library's device image, so it must give the same answer
as schur_refine_residuals and as the oracle's double-double residuals, call
after call, even though every call reuses the array the previous one left
behind, and it must take no device memory of its own. This file is collected
last on purpose.
"""
import numpy as np
import pytest

from paper_2203_10879_gb300 import _binding as B
from paper_2203_10879_gb300 import inputs
import oracle
from gpu_util import to_dev

pytestmark = pytest.mark.gpu


def _with_handle(n, A, Q):
    s, h = B.schur_refine_create(n, B.default_options(), None)
    assert s == B.SR_OK
    try:
        s, rT, rQ = B.schur_refine_residuals(h, n, A, Q)
        assert s == B.SR_OK
        return rT, rQ
    finally:
        B.schur_refine_destroy(h)


def test_noalloc_residuals_match_oracle_and_handle_entry_point_twice():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    stream = torch.cuda.current_stream().cuda_stream
    # two problems, all device inputs made before the first call
    cases = []
    for n, seed in ((512, 3), (200, 4)):
        p = inputs.planted(n, inputs.eig_unit_step(n), seed, pert=1e-6)
        Q, _ = oracle.ns_init(p.Qhat)
        cases.append((n, p.A, Q, to_dev(p.A), to_dev(Q)))
    torch.cuda.synchronize()
    got = []
    free = []
    # two calls in a row on different problems: the second must not see the
    # first's scratch, and neither may take device memory (the first call on
    # the device may load the module; the second must change nothing)
    for n, _, _, A_d, Q_d in cases:
        s, rT, rQ = B.schur_refine_residuals_noalloc(n, A_d, Q_d, stream)
        assert s == B.SR_OK
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        got.append((rT, rQ))
    assert free[1] == free[0]
    for (n, A, Q, A_d, Q_d), (rT, rQ) in zip(cases, got):
        assert np.isfinite(rT) and np.isfinite(rQ) and rT > 0
        # the oracle's double-double residuals of the same A and Q
        oT, oQ = oracle.residuals_dd(A, Q)
        assert rT == pytest.approx(oT, rel=1e-8)
        assert rQ == pytest.approx(oQ, rel=1e-6, abs=1e-18)
        # and the handle-based entry point (same tolerance as the residual parity tests)
        hT, hQ = _with_handle(n, A_d, Q_d)
        assert rT == pytest.approx(hT, rel=1e-8)
        assert rQ == pytest.approx(hQ, rel=1e-6, abs=1e-18)


def test_noalloc_zero_matrix_gives_zero_relative_residual():
    torch = pytest.importorskip("torch")
    n = 48
    Q = np.linalg.qr(np.random.default_rng(5).standard_normal((n, n)))[0]
    s, rT, rQ = B.schur_refine_residuals_noalloc(n, to_dev(np.zeros((n, n))), to_dev(Q),
                                                 torch.cuda.current_stream().cuda_stream)
    assert s == B.SR_OK
    assert rT == 0.0
    assert rQ == pytest.approx(oracle.residuals_dd(np.eye(n), Q)[1], rel=1e-6, abs=1e-18)


def test_noalloc_rejects_orders_above_its_scratch():
    torch = pytest.importorskip("torch")
    n = 513
    A = to_dev(np.eye(n))
    s, _, _ = B.schur_refine_residuals_noalloc(n, A, A, torch.cuda.current_stream().cuda_stream)
    assert s == B.SR_ERR_INVALID_ARG
