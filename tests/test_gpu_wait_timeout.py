"""The dataflow solve's waits are bounded: a wait whose tile is never
published gives up, the kernel reports SR_FLAG_TIMEOUT and returns, and the
handle and its CUDA context stay usable (no fault, no hang)."""
import time

import numpy as np
import pytest

import oracle
from paper_2203_10879_gb300 import _binding as B
from gpu_util import from_dev, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    B.lib()
    return torch


def test_unsatisfiable_wait_times_out_and_context_survives(torch):
    s, h = B.schur_refine_create(128, B.default_options(lp=B.SR_LP_FP32), None)
    assert s == B.SR_OK
    try:
        t0 = time.perf_counter()
        assert B.schur_refine_selftest_wait_timeout(h) == B.SR_ERR_TIMEOUT
        assert time.perf_counter() - t0 < 30.0   # one bounded wait (about a second)
        # the same handle solves a well-posed problem afterwards
        n = 100
        rng = np.random.default_rng(5)
        d = np.arange(n, dtype=float) / 4.0 + rng.uniform(0, 0.1, n)
        T = np.triu(rng.standard_normal((n, n)) * 0.05, 1) + np.diag(d)
        E = np.tril(rng.standard_normal((n, n)) * 1e-3, -1)
        TE = to_dev((np.triu(T) + E).astype(np.float32))
        assert B.schur_refine_trisolve(h, n, TE, to_dev(d.copy())) == B.SR_OK
        L = np.tril(from_dev(TE), -1).astype(np.float64)
        ref = oracle.alg2(T, E, d)
        assert np.linalg.norm(L - ref) <= 1e-5 * np.linalg.norm(ref)
        torch.cuda.synchronize()
    finally:
        B.schur_refine_destroy(h)
