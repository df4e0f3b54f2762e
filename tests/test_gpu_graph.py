"""Graph mode of schur_refine_step (option graph = 1): the whole call is one CUDA
graph whose REPEAT loop and stop test run on the device (conditional WHILE and
IF nodes). It replays the same kernels on the same data as the host-driven
loop, so statuses, counters and the refined factor must agree bit for bit,
including on the failure path and when the graph is rebuilt for new buffers.
"""
import numpy as np
import pytest

import oracle
from paper_2203_10879_gb300 import _binding as B
from paper_2203_10879_gb300 import inputs
from gpu_util import from_dev, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available()
    B.lib()
    return torch


def _run(torch, p, graph, repeats=1, **kw):
    s, h = B.schur_refine_create(p.n, B.default_options(graph=graph, **kw), None)
    assert s == B.SR_OK, B.status_string(s)
    try:
        A = to_dev(p.A)
        Qh = to_dev(p.Qhat)
        res = []
        for _ in range(repeats):
            Q = torch.zeros((p.n, p.n), dtype=torch.float64, device="cuda").t()
            T = torch.zeros((p.n, p.n), dtype=torch.float64, device="cuda").t()
            st, nr = B.schur_refine_step(h, p.n, A, Q, Qh, T)
            res.append((st, nr.iters, nr.hp_gemms, nr.stril_rel, nr.orth, from_dev(Q), from_dev(T)))
        return res
    finally:
        B.schur_refine_destroy(h)


CASES = [
    ("all-FP64 n=64", lambda: inputs.unit_step_real(64), dict(hp_gemm=B.SR_HP_FP64, lp=B.SR_LP_FP64)),
    ("mixed native n=100", lambda: inputs.jittered_real(100), dict(hp_gemm=B.SR_HP_FP64, lp=B.SR_LP_FP32)),
    ("mixed emulated n=300", lambda: inputs.jittered_real(300), dict(hp_gemm=B.SR_HP_OZAKI_BF16, lp=B.SR_LP_FP32)),
    ("emulated full sigma n=97", lambda: inputs.unit_step_real(97),
     dict(hp_gemm=B.SR_HP_OZAKI_BF16, lp=B.SR_LP_FP32, full_sigma=1)),
]


@pytest.mark.parametrize("name,make,kw", CASES, ids=[c[0] for c in CASES])
def test_graph_mode_equals_host_loop(torch, name, make, kw):
    p = make()
    host = _run(torch, p, 0, **kw)[0]
    g = _run(torch, p, 1, repeats=3, **kw)   # built once, replayed twice (new Q buffers: rebuilt)
    for r in g:
        assert r[:3] == host[:3], name
        assert r[3] == host[3] and r[4] == host[4]
        assert np.array_equal(r[5], host[5]) and np.array_equal(r[6], host[6])
    assert host[0] == B.SR_OK
    tol = oracle.default_tol(p.n)
    cT, cQ = oracle.residuals_dd(p.A, g[0][5])
    assert cT <= tol and cQ <= tol


def test_graph_mode_failure_path_and_max_iter(torch):
    bad = inputs.jittered_real(200, upper_std=1.0 / np.sqrt(200))
    kw = dict(hp_gemm=B.SR_HP_OZAKI_BF16, lp=B.SR_LP_FP32)
    h0 = _run(torch, bad, 0, **kw)[0]
    g0 = _run(torch, bad, 1, **kw)[0]
    assert h0[0] in (B.SR_ERR_NONFINITE, B.SR_ERR_NOT_CONVERGED, B.SR_ERR_NONDISTINCT)
    assert g0[:3] == h0[:3]
    p = inputs.jittered_real(128)
    h1 = _run(torch, p, 0, max_iter=1, **kw)[0]
    g1 = _run(torch, p, 1, max_iter=1, **kw)[0]
    assert h1[0] == B.SR_ERR_NOT_CONVERGED and g1[:3] == h1[:3]
    assert np.array_equal(g1[5], h1[5])


def test_graph_mode_replay_same_buffers(torch):
    p = inputs.unit_step_real(64)
    s, h = B.schur_refine_create(64, B.default_options(graph=1, hp_gemm=B.SR_HP_FP64, lp=B.SR_LP_FP64), None)
    assert s == B.SR_OK
    try:
        A, Qh = to_dev(p.A), to_dev(p.Qhat)
        Q = torch.zeros((64, 64), dtype=torch.float64, device="cuda").t()
        out = []
        for _ in range(4):
            st, nr = B.schur_refine_step(h, 64, A, Q, Qh)
            assert st == B.SR_OK
            out.append(from_dev(Q))
        assert all(np.array_equal(out[0], q) for q in out[1:])
    finally:
        B.schur_refine_destroy(h)
