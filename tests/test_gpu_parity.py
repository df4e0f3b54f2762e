"""GPU parity: the CUDA library, called through its C ABI, against the CPU oracle.

Tolerances follow from the arithmetic:
  * a product of depth k in FP64 carries entrywise error <= k u |A||B| (u = 2^-53);
  * the triangular solve in FP64 agrees with Alg. 2 to a few hundred u times the
    size of L on the well-separated test spectra used here; in FP32 both the
    GPU and the oracle are off the FP64 solution by O(u32 |L|), so the GPU's
    error is compared with the oracle's own FP32 error;
  * refined factors are checked by the target itself: residuals certified in
    double-double <= 1e-14 sqrt(n), diagonal of T against the oracle, columns of
    Q against the oracle and the planted Q0 up to sign where eigenvalue gaps
    are >= 1e-2 (1e-12).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2203_10879_gb300 import _binding as B
from paper_2203_10879_gb300 import inputs
from gpu_util import from_dev, phase_align, sign_align, to_dev

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    B.lib()
    return torch


def _handle(n_max, **kw):
    s, h = B.schur_refine_create(n_max, B.default_options(**kw), None)
    assert s == B.SR_OK, B.status_string(s)
    return h


# ---------------------------------------------------------------------------
# high-precision products

@pytest.mark.parametrize("m,n,k", [(64, 64, 64), (100, 77, 129), (257, 33, 300), (1, 5, 3)])
@pytest.mark.parametrize("transA", [0, 1])
def test_hp_gemm_native_parity(torch, m, n, k, transA):
    rng = np.random.default_rng(m * 1000 + n + k)
    A = rng.standard_normal((k, m) if transA else (m, k))
    Bm = rng.standard_normal((k, n))
    h = _handle(max(m, n, k))
    try:
        C = torch.zeros((n, m), dtype=torch.float64, device="cuda").t()
        s = B.schur_refine_gemm(h, transA, m, n, k, to_dev(A), to_dev(Bm), C)
        assert s == B.SR_OK
        opA = A.T if transA else A
        ref = opA @ Bm
        bound = 2 * k * U64 * (np.abs(opA) @ np.abs(Bm)) + 1e-300
        assert np.all(np.abs(from_dev(C) - ref) <= bound)
    finally:
        B.schur_refine_destroy(h)


# ---------------------------------------------------------------------------
# triangular matrix equation

def _solve_problem(n, seed):
    rng = np.random.default_rng(seed)
    d = np.arange(n, dtype=float) / 4.0 + rng.uniform(0, 0.1, n)
    T = np.triu(rng.standard_normal((n, n)) * 0.05, 1) + np.diag(d)
    E = np.tril(rng.standard_normal((n, n)) * 1e-3, -1)
    return T, E


SOLVE_MODES = [1, 2]   # one dataflow launch; one launch pair per block subdiagonal


@pytest.mark.parametrize("solve_mode", SOLVE_MODES)
@pytest.mark.parametrize("n", [1, 2, 5, 31, 32, 33, 64, 100, 257, 700])
def test_trisolve_fp64_parity(torch, n, solve_mode):
    T, E = _solve_problem(n, n)
    h = _handle(n, lp=B.SR_LP_FP64, solve_mode=solve_mode)
    try:
        TE = to_dev(np.triu(T) + E)
        s = B.schur_refine_trisolve(h, n, TE, to_dev(np.diagonal(T).copy()))
        assert s == B.SR_OK
        out = from_dev(TE)
        L = np.tril(out, -1)
        assert np.array_equal(np.triu(out), np.triu(T))     # upper triangle untouched
        ref = oracle.alg2(T, E, np.diagonal(T).copy())
        scale = max(np.max(np.abs(ref)), 1e-300)
        assert np.max(np.abs(L - ref)) <= 1e3 * U64 * scale
    finally:
        B.schur_refine_destroy(h)


@pytest.mark.parametrize("solve_mode", SOLVE_MODES)
@pytest.mark.parametrize("n", [2, 33, 100, 257, 700, 1000])
def test_trisolve_fp32_parity(torch, n, solve_mode):
    T, E = _solve_problem(n, 7 * n)
    h = _handle(n, lp=B.SR_LP_FP32, solve_mode=solve_mode)
    try:
        TE = to_dev((np.triu(T) + E).astype(np.float32))
        s = B.schur_refine_trisolve(h, n, TE, to_dev(np.diagonal(T).copy()))
        assert s == B.SR_OK
        L32 = np.tril(from_dev(TE), -1).astype(np.float64)
        L64 = oracle.alg2(T, E, np.diagonal(T).copy())
        Lo32 = oracle.alg2(np.triu(T).astype(np.float32), E.astype(np.float32), np.diagonal(T).copy())
        e_gpu = np.linalg.norm(L32 - L64)
        e_orc = np.linalg.norm(Lo32.astype(np.float64) - L64)
        # both forms sum each tile's block products apart from E and add E once
        # (as Alg. 2 adds e_ij once after the two sums)
        assert e_gpu <= 10 * max(e_orc, U32 * np.linalg.norm(L64))
    finally:
        B.schur_refine_destroy(h)


@pytest.mark.parametrize("solve_mode", SOLVE_MODES)
@pytest.mark.parametrize("lp", [B.SR_LP_FP32, B.SR_LP_FP64])
def test_trisolve_equal_diagonal_reports_nondistinct(torch, lp, solve_mode):
    n = 40
    T, E = _solve_problem(n, 3)
    T[30, 30] = T[3, 3]
    dt = np.float32 if lp == B.SR_LP_FP32 else np.float64
    h = _handle(n, lp=lp, solve_mode=solve_mode)
    try:
        s = B.schur_refine_trisolve(h, n, to_dev((np.triu(T) + E).astype(dt)), to_dev(np.diagonal(T).copy()))
        assert s == B.SR_ERR_NONDISTINCT
    finally:
        B.schur_refine_destroy(h)


@pytest.mark.parametrize("lp", [B.SR_LP_FP32, B.SR_LP_FP64])
def test_trisolve_modes_agree(torch, lp):
    """Both launch forms solve the same tile equations: on a ragged order
    spanning many tiles they agree to the working precision's rounding."""
    n = 1000
    T, E = _solve_problem(n, 11)
    dt = np.float32 if lp == B.SR_LP_FP32 else np.float64
    u = U32 if lp == B.SR_LP_FP32 else U64
    out = []
    for mode in SOLVE_MODES:
        h = _handle(n, lp=lp, solve_mode=mode)
        try:
            TE = to_dev((np.triu(T) + E).astype(dt))
            assert B.schur_refine_trisolve(h, n, TE, to_dev(np.diagonal(T).copy())) == B.SR_OK
            out.append(np.tril(from_dev(TE), -1).astype(np.float64))
        finally:
            B.schur_refine_destroy(h)
    assert np.linalg.norm(out[0] - out[1]) <= 100 * u * np.linalg.norm(out[1])


# ---------------------------------------------------------------------------
# the whole iteration

def _refine_gpu(p, **kw):
    import torch
    n = p.n
    h = _handle(n, **kw)
    try:
        A = to_dev(p.A)
        Qhat = to_dev(p.Qhat)
        dt = torch.complex128 if np.iscomplexobj(p.A) else torch.float64
        Q = torch.zeros((n, n), dtype=dt, device="cuda").t()
        T = torch.zeros((n, n), dtype=dt, device="cuda").t()
        s, nr = B.schur_refine_step(h, n, A, Q, Qhat, T)
        sr, rT, rQ = B.schur_refine_residuals(h, n, A, Q)
        assert sr == B.SR_OK
        return s, nr, from_dev(Q), from_dev(T), (rT, rQ)
    finally:
        B.schur_refine_destroy(h)


def test_refine_unit_step_n64_all_fp64(torch):
    p = inputs.unit_step_real(64)
    s, nr, Q, T, (rT, rQ) = _refine_gpu(p, lp=B.SR_LP_FP64)
    ref = oracle.refine(p.A, p.Qhat, lp="f64")
    assert s == B.SR_OK and ref.status == oracle.OK
    assert nr.iters == ref.iters and nr.hp_gemms == 4 * nr.iters
    tol = oracle.default_tol(64)
    cT, cQ = oracle.residuals_dd(p.A, Q)
    assert cT <= tol and cQ <= tol
    assert rT == pytest.approx(cT, rel=1e-6, abs=1e-18)
    assert rQ == pytest.approx(cQ, rel=1e-6, abs=1e-18)
    assert np.max(np.abs(sign_align(Q, ref.Q) - ref.Q)) <= 1e-12
    assert np.max(np.abs(sign_align(Q, p.Q0) - p.Q0)) <= 1e-12      # gaps 1/64 >= 1e-2
    assert np.max(np.abs(np.diagonal(T) - p.lam)) <= 1e-12


@pytest.mark.parametrize("solve_mode", SOLVE_MODES)
@pytest.mark.parametrize("lp", [B.SR_LP_FP32, B.SR_LP_FP64])
def test_refine_jittered_ragged(torch, lp, solve_mode):
    n = 300   # not a multiple of any tile size
    p = inputs.jittered_real(n)
    s, nr, Q, T, (rT, rQ) = _refine_gpu(p, lp=lp, solve_mode=solve_mode)
    ref = oracle.refine(p.A, p.Qhat, lp="f32" if lp == B.SR_LP_FP32 else "f64")
    assert s == B.SR_OK
    assert abs(nr.iters - ref.iters) <= 1
    tol = oracle.default_tol(n)
    cT, cQ = oracle.residuals_dd(p.A, Q)
    assert cT <= tol and cQ <= tol
    Tref = ref.Q.T @ p.A @ ref.Q
    assert np.max(np.abs(np.diagonal(T) - np.diagonal(Tref))) <= 1e-12
    assert np.max(np.abs(sign_align(Q, ref.Q) - ref.Q)) <= 1e-9


@pytest.mark.parametrize("lp,qtol", [(B.SR_LP_FP64, 1e-13), (B.SR_LP_FP32, None)])
def test_one_pass_parity(torch, lp, qtol):
    p = inputs.planted(96, inputs.eig_unit_step(96), 5, pert=1e-5)
    s, nr, Q, T, _ = _refine_gpu(p, lp=lp, max_iter=1)
    assert s == B.SR_ERR_NOT_CONVERGED and nr.iters == 1
    Q0, y0 = oracle.ns_init(p.Qhat)
    parts = {}
    Q1, info = oracle.iteration(p.A, Q0, lp="f64" if lp == B.SR_LP_FP64 else "f32", parts=parts)
    assert nr.orth == pytest.approx(info.y_norm, rel=1e-3, abs=96 * U64)   # rounding-level quantity
    assert nr.w_norm == pytest.approx(info.w_norm, rel=1e-5)
    if qtol is None:   # FP32 solve: L agrees to O(u32) relative, so Q to O(u32 ||W||)
        qtol = 50 * U32 * info.w_norm + 1e-13
    assert np.max(np.abs(Q - Q1)) <= qtol


@pytest.mark.parametrize("n", [64, 200])
def test_residuals_parity(torch, n):
    p = inputs.unit_step_real(n)
    Q, _ = oracle.ns_init(p.Qhat)
    h = _handle(n)
    try:
        s, rT, rQ = B.schur_refine_residuals(h, n, to_dev(p.A), to_dev(Q))
        assert s == B.SR_OK
    finally:
        B.schur_refine_destroy(h)
    cT, cQ = oracle.residuals_dd(p.A, Q)
    assert rT == pytest.approx(cT, rel=1e-8)
    assert rQ == pytest.approx(cQ, rel=1e-6, abs=1e-18)


def test_failure_path_reports_status(torch):
    p = inputs.jittered_real(128, upper_std=1 / math.sqrt(128))
    s, nr, Q, T, _ = _refine_gpu(p, lp=B.SR_LP_FP32, max_iter=10)
    assert s in (B.SR_ERR_NONFINITE, B.SR_ERR_NOT_CONVERGED, B.SR_ERR_NONDISTINCT)
    assert nr.iters <= 10


def test_step_rejects_order_above_n_max(torch):
    h = _handle(16)
    try:
        A = to_dev(np.eye(32))
        s, _ = B.schur_refine_step(h, 32, A, to_dev(np.eye(32)))
        assert s == B.SR_ERR_INVALID_ARG
    finally:
        B.schur_refine_destroy(h)


def test_profile_counts(torch):
    p = inputs.unit_step_real(64)
    h = _handle(64, lp=B.SR_LP_FP64, profile=1)
    try:
        import torch as T
        Q = T.zeros((64, 64), dtype=T.float64, device="cuda").t()
        s, nr = B.schur_refine_step(h, 64, to_dev(p.A), Q, to_dev(p.Qhat))
        assert s == B.SR_OK
        s, prof = B.schur_refine_get_profile(h)
        d = prof.as_dict()
        assert d["hp_gemm"]["launches"] == nr.hp_gemms
        assert d["hp_gemm"]["flops"] == nr.hp_gemms * 2 * 64 ** 3
        assert d["hp_gemm"]["ms"] > 0 and d["solve"]["ms"] > 0
    finally:
        B.schur_refine_destroy(h)


# ---------------------------------------------------------------------------
# symmetric A (Sec. 2.5)

@pytest.mark.parametrize("lp,dt", [(B.SR_LP_FP32, np.float32), (B.SR_LP_FP64, np.float64)])
@pytest.mark.parametrize("n", [1, 2, 33, 257])
def test_symmetric_solve_bit_exact(torch, n, lp, dt):
    """T diagonal: the GPU's elementwise solve performs the oracle's operations
    (divisor from the FP64 diagonal rounded once, one IEEE division)."""
    rng = np.random.default_rng(n)
    d = np.sort(rng.uniform(-1.0, 1.0, n))
    E = np.tril(rng.standard_normal((n, n)) * 1e-4, -1)
    h = _handle(n, lp=lp, symmetric=1)
    try:
        TE = to_dev((np.diag(d) + np.triu(rng.standard_normal((n, n)), 1) + E).astype(dt))
        assert B.schur_refine_trisolve(h, n, TE, to_dev(d.copy())) == B.SR_OK
        L = np.tril(from_dev(TE), -1)
        ref = oracle.sym_solve(E.astype(dt), d)
        assert np.array_equal(L, ref)
    finally:
        B.schur_refine_destroy(h)


def test_symmetric_solve_reports_equal_diagonal(torch):
    n = 40
    d = np.linspace(0.0, 1.0, n)
    d[30] = d[3]
    h = _handle(n, lp=B.SR_LP_FP32, symmetric=1)
    try:
        TE = to_dev((np.diag(d) + np.tril(np.ones((n, n)) * 1e-3, -1)).astype(np.float32))
        assert B.schur_refine_trisolve(h, n, TE, to_dev(d.copy())) == B.SR_ERR_NONDISTINCT
    finally:
        B.schur_refine_destroy(h)


@pytest.mark.parametrize("hp", [B.SR_HP_FP64, B.SR_HP_OZAKI_BF16])
@pytest.mark.parametrize("n", [64, 300])
def test_symmetric_refinement_parity(torch, n, hp):
    p = inputs.symmetric_real(n)
    s, nr, Q, T, (rT, rQ) = _refine_gpu(p, lp=B.SR_LP_FP32, hp_gemm=hp, symmetric=1)
    ref = oracle.refine(p.A, p.Qhat, lp="f32", symmetric=True)
    assert s == B.SR_OK and ref.status == oracle.OK
    assert abs(nr.iters - ref.iters) <= 1
    tol = oracle.default_tol(n)
    cT, cQ = oracle.residuals_dd(p.A, Q)
    assert cT <= tol and cQ <= tol
    w, V = np.linalg.eigh(p.A)
    assert np.max(np.abs(np.diagonal(T) - w)) <= 1e-13
    assert np.max(np.abs(sign_align(Q, V) - V)) <= 1e-10
    assert np.max(np.abs(sign_align(Q, ref.Q) - ref.Q)) <= 1e-10


def test_symmetric_option_rejected_for_dd(torch):
    kw = {"target": B.SR_TARGET_DD, "lp": B.SR_LP_FP64, "qhat_type": B.SR_QHAT_FP64}
    s, h = B.schur_refine_create(64, B.default_options(symmetric=1, **kw), None)
    assert s == B.SR_ERR_UNSUPPORTED and not h


# Hermitian A (Sec. 2.5 for complex data): the divisor from the real parts of
# the hp diagonal, rounded once to FP32, dividing both parts of e_ij

@pytest.mark.parametrize("n", [2, 33, 257])
def test_hermitian_solve_bit_exact(torch, n):
    rng = np.random.default_rng(3 * n)
    d = np.sort(rng.uniform(-1.0, 1.0, n)) + 1j * rng.uniform(-1e-17, 1e-17, n)   # rounding-level imaginary parts
    E = np.tril(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)), -1) * 1e-4
    h = _handle(n, dtype=B.SR_COMPLEX, hp_gemm=B.SR_HP_OZAKI_CRT, lp=B.SR_LP_FP32, symmetric=1)
    try:
        U = np.triu(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)), 1)
        TE = to_dev((np.diag(d) + U + E).astype(np.complex64))
        assert B.schur_refine_trisolve(h, n, TE, to_dev(d.copy())) == B.SR_OK
        L = np.tril(from_dev(TE), -1)
        ref = oracle.sym_solve(E.astype(np.complex64), d)
        assert np.array_equal(L, ref)
    finally:
        B.schur_refine_destroy(h)


@pytest.mark.parametrize("hp", [B.SR_HP_OZAKI_CRT, B.SR_HP_OZAKI_BF16])
@pytest.mark.parametrize("n", [64, 300])
def test_hermitian_refinement_parity(torch, n, hp):
    p = inputs.hermitian_complex(n)
    s, nr, Q, T, (rT, rQ) = _refine_gpu(p, lp=B.SR_LP_FP32, hp_gemm=hp, symmetric=1, dtype=B.SR_COMPLEX)
    ref = oracle.refine(p.A, p.Qhat, lp="f32", symmetric=True)
    assert s == B.SR_OK and ref.status == oracle.OK
    assert abs(nr.iters - ref.iters) <= 1
    tol = oracle.default_tol(n)
    cT, cQ = oracle.residuals_dd(p.A, Q)
    assert cT <= tol and cQ <= tol
    w, V = np.linalg.eigh(p.A)
    assert np.max(np.abs(np.diagonal(T) - w)) <= 1e-13
    assert np.max(np.abs(phase_align(Q, V) - V)) <= 1e-10
    assert np.max(np.abs(phase_align(Q, ref.Q) - ref.Q)) <= 1e-10


# ---------------------------------------------------------------------------
# entry threshold of Example 4 (Sec. 3)

def _threshold_problem(n, seed):
    """Evenly spaced eigenvalues k/n with weak coupling (|t_ij| ~ 0.1/n), except
    a cluster of six 1e-9 apart: the entries of L inside the cluster are ~1e-3
    and feed one another, every other entry is below ~1e-8, so GPU and oracle
    take the same clamp decisions whatever the order of their sums."""
    rng = np.random.default_rng(seed)
    d = np.arange(n, dtype=np.float64) / n
    k = n // 2
    d[k - 5:k + 1] = d[k - 5] + 1e-9 * np.arange(6)
    T = np.triu(rng.standard_normal((n, n)) * (0.1 / n), 1) + np.diag(d)
    g = rng.standard_normal((n, n))
    E = np.tril(np.sign(g) * (1.0 + np.abs(g)) * 1e-12, -1)   # |e_ij| >= 1e-12
    return T, E, d


@pytest.mark.parametrize("solve_mode", SOLVE_MODES)
@pytest.mark.parametrize("lp,dt,rtol", [(B.SR_LP_FP32, np.float32, 1e-4), (B.SR_LP_FP64, np.float64, 1e-12)])
@pytest.mark.parametrize("n", [33, 100, 257])
def test_trisolve_threshold_parity(torch, n, lp, dt, rtol, solve_mode):
    T, E, d = _threshold_problem(n, 3 * n)
    h = _handle(n, lp=lp, solve_mode=solve_mode, l_cap=1e-5)
    try:
        TE = to_dev((np.triu(T) + E).astype(dt))
        assert B.schur_refine_trisolve(h, n, TE, to_dev(d.copy())) == B.SR_OK
        L = np.tril(from_dev(TE), -1).astype(np.float64)
    finally:
        B.schur_refine_destroy(h)
    ref = oracle.alg2(np.triu(T).astype(dt), E.astype(dt), d, 1e-5).astype(np.float64)
    free = oracle.alg2(np.triu(T).astype(dt), E.astype(dt), d).astype(np.float64)
    assert np.max(np.abs(free)) > 1e-4                     # the cluster's entries exceed the threshold
    assert np.max(np.abs(ref)) < 1e-7 and np.max(np.abs(L)) < 1e-7
    assert np.array_equal(np.tril(L == 0, -1), np.tril(ref == 0, -1))
    assert np.linalg.norm(L - ref) <= rtol * np.linalg.norm(ref)


@pytest.mark.parametrize("lp,dt", [(B.SR_LP_FP32, np.float32), (B.SR_LP_FP64, np.float64)])
def test_symmetric_solve_threshold_bit_exact(torch, lp, dt):
    n = 64
    rng = np.random.default_rng(4)
    d = np.sort(rng.uniform(0.0, 1.0, n))
    d[10] = d[9] + 1e-9
    E = np.tril(rng.standard_normal((n, n)) * 1e-12, -1)
    h = _handle(n, lp=lp, symmetric=1, l_cap=1e-5)
    try:
        TE = to_dev((np.diag(d) + E).astype(dt))
        assert B.schur_refine_trisolve(h, n, TE, to_dev(d.copy())) == B.SR_OK
        L = np.tril(from_dev(TE), -1)
    finally:
        B.schur_refine_destroy(h)
    ref = oracle.sym_solve(E.astype(dt), d, 1e-5)
    assert ref[10, 9] == 0 and np.array_equal(L, ref)
