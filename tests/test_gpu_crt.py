"""GPU parity of the residue form of the emulated products (SR_HP_OZAKI_CRT)
and of the refinement that uses it, through the C ABI, against the oracle.

The bound used below is fixed by the definition of the form, computed here
with Python integers (not by the library): the moduli are the N largest
pairwise coprime integers <= 256 taken greedily, M their product, and t the
largest integer with k 2^(2t) < M / 2. Every entry x of a row of op(A) (column
of B) with scale 2^e (|x| < 2^e) becomes round(x 2^(t-e)), an error of at most
2^(e-t-1); so per term |ab - emulated| <= 2^(e_i + f_j - t) (1 + 2^-t), over
k terms |C - AB| <= k 2^(e_i + f_j - t) (1 + 2^-t), plus the one rounding of
the rebuilt value to FP64 (u |C|). Integer operands of fewer than t bits are
held exactly, and so is every product: bit-exact results.
"""
from math import gcd

import numpy as np
import pytest

import oracle
from paper_2203_10879_gb300 import _binding as B
from paper_2203_10879_gb300 import inputs
from gpu_util import from_dev, phase_align, sign_align, to_dev

pytestmark = pytest.mark.gpu
U64 = 2.0 ** -53
U32 = 2.0 ** -24


def moduli(N):
    ms = []
    m = 256
    while len(ms) < N:
        if all(gcd(m, x) == 1 for x in ms):
            ms.append(m)
        m -= 1
    return ms


def bits_t(N, k):
    M = 1
    for m in moduli(N):
        M *= m
    t = 0
    while k * 2 ** (2 * (t + 1)) * 2 < M:
        t += 1
    return t


def test_moduli_and_bits_follow_the_definition():
    # the 16 moduli and the bits they give at the inner lengths of the workloads
    assert moduli(16) == [256, 255, 253, 251, 247, 241, 239, 233, 229, 227, 223, 217, 211, 199, 197, 193]
    assert [bits_t(16, k) for k in (64, 4096, 8192, 16384)] == [59, 56, 55, 55]
    assert bits_t(32, 2048) == 114


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available()
    B.lib()
    return torch


def _gemm(torch, A, Bm, transA, N=0, cplx=False):
    m = A.shape[1] if transA else A.shape[0]
    k = A.shape[0] if transA else A.shape[1]
    n = Bm.shape[1]
    kw = dict(hp_gemm=B.SR_HP_OZAKI_CRT, ozaki_slices=N)
    if cplx:
        kw.update(dtype=B.SR_COMPLEX, lp=B.SR_LP_FP32)
    s, h = B.schur_refine_create(max(m, n, k), B.default_options(**kw), None)
    assert s == B.SR_OK, B.status_string(s)
    try:
        C = torch.zeros((n, m), dtype=torch.complex128 if cplx else torch.float64, device="cuda").t()
        st = B.schur_refine_gemm(h, int(transA), m, n, k, to_dev(A), to_dev(Bm), C)
        assert st == B.SR_OK, B.status_string(st)
        return from_dev(C)
    finally:
        B.schur_refine_destroy(h)


def test_crt_options_gate(torch):
    # FP64 results hold M in 128 bits: at most 16 moduli
    s, h = B.schur_refine_create(64, B.default_options(hp_gemm=B.SR_HP_OZAKI_CRT, ozaki_slices=17), None)
    assert s == B.SR_ERR_INVALID_ARG and not h.value


def test_crt_single_tile_exact_integers(torch):
    rng = np.random.default_rng(1)
    A = rng.integers(-100, 101, (128, 256)).astype(np.float64)
    Bm = rng.integers(-100, 101, (256, 128)).astype(np.float64)
    assert np.array_equal(_gemm(torch, A, Bm, False), A @ Bm)


@pytest.mark.parametrize("m,n,k,transA", [(200, 130, 300, False), (129, 257, 513, True), (1, 3, 2, False),
                                          (300, 300, 1000, False)])
def test_crt_exact_integers_ragged(torch, m, n, k, transA):
    # 2^20-sized integers: the products reach 2^50 k, far beyond what the
    # moduli hold one at a time, so every residue and the rebuild take part
    rng = np.random.default_rng(m + n + k)
    A = rng.integers(-2 ** 20, 2 ** 20, (k, m) if transA else (m, k)).astype(np.float64)
    Bm = rng.integers(-2 ** 20, 2 ** 20, (k, n)).astype(np.float64)
    opA = A.T if transA else A
    C = _gemm(torch, A, Bm, transA)
    ref = (opA.astype(object) @ Bm.astype(object))      # exact Python integers
    assert np.array_equal(C, np.array(ref, dtype=np.float64))


def _scales(X, axis):
    return np.ceil(np.log2(np.max(np.abs(X), axis=axis) * (1 + 2 ** -52)))


@pytest.mark.parametrize("N", [16, 12, 8])
@pytest.mark.parametrize("m,n,k,transA", [(160, 96, 700, True), (300, 300, 300, False)])
def test_crt_error_law(torch, N, m, n, k, transA):
    rng = np.random.default_rng(7 * m + k + N)
    A = rng.standard_normal((k, m) if transA else (m, k)) * np.exp(rng.uniform(-3, 3, (1, m) if transA else (m, 1)))
    Bm = rng.standard_normal((k, n))
    C = _gemm(torch, A, Bm, transA, N=N)
    hi, lo = oracle.gemm_dd(A, None, Bm, None, transA=transA)
    opA = A.T if transA else A
    t = bits_t(N, k)
    scale = 2.0 ** (_scales(opA, 1)[:, None] + _scales(Bm, 0)[None, :])
    bound = k * scale * 2.0 ** -t * (1 + 2.0 ** -t) + U64 * np.abs(hi)
    err = np.abs(C - hi - lo)
    assert np.all(err <= bound)
    if N == 16:
        # at 16 moduli the product meets the FP64 bound k u |A||B| with room to spare
        assert np.all(err <= k * U64 * (np.abs(opA) @ np.abs(Bm)))
    else:
        assert np.max(err / bound) > 1e-4   # fewer moduli really truncate: not secretly exact


def test_crt_nonfinite_input_gives_nan(torch):
    A = np.ones((64, 64))
    A[5, 7] = np.inf
    C = _gemm(torch, A, np.ones((64, 64)), False)
    assert np.all(np.isnan(C[5, :]))
    assert np.all(np.isfinite(np.delete(C, 5, axis=0)))


@pytest.mark.parametrize("m,n,k,transA", [(96, 70, 130, True), (200, 64, 300, False)])
def test_crt_complex_gemm_accuracy(torch, m, n, k, transA):
    rng = np.random.default_rng(m + k)
    shpA = (k, m) if transA else (m, k)
    A = rng.standard_normal(shpA) + 1j * rng.standard_normal(shpA)
    Bm = rng.standard_normal((k, n)) + 1j * rng.standard_normal((k, n))
    C = _gemm(torch, A, Bm, transA, cplx=True)
    opA = A.conj().T if transA else A
    # each part is a real product of depth 2k over the stacked [re, im] vectors
    Ar, Ai, Br, Bi = opA.real, opA.imag, Bm.real, Bm.imag
    rr = oracle.gemm_dd(np.hstack([Ar, -Ai]), None, np.vstack([Br, Bi]), None)
    ri = oracle.gemm_dd(np.hstack([Ar, Ai]), None, np.vstack([Bi, Br]), None)
    mag = (np.abs(Ar) + np.abs(Ai)) @ (np.abs(Br) + np.abs(Bi))
    bound = 2 * k * U64 * mag
    assert np.all(np.abs(C.real - rr[0] - rr[1]) <= bound)
    assert np.all(np.abs(C.imag - ri[0] - ri[1]) <= bound)


# ---------------------------------------------------------------------------
# refinement with the residue form

def _refine(p, cplx=False, T=False, **kw):
    import torch
    n = p.n
    opt = dict(hp_gemm=B.SR_HP_OZAKI_CRT, lp=B.SR_LP_FP32)
    if cplx:
        opt["dtype"] = B.SR_COMPLEX
    opt.update(kw)
    s, h = B.schur_refine_create(n, B.default_options(**opt), None)
    assert s == B.SR_OK
    dt = torch.complex128 if cplx else torch.float64
    try:
        Q = torch.zeros((n, n), dtype=dt, device="cuda").t()
        Td = torch.zeros((n, n), dtype=dt, device="cuda").t() if T else None
        st, nr = B.schur_refine_step(h, n, to_dev(p.A), Q, to_dev(p.Qhat), Td)
        return st, nr, from_dev(Q), (from_dev(Td) if T else None)
    finally:
        B.schur_refine_destroy(h)


def test_crt_refine_unit_step_n64(torch):
    p = inputs.unit_step_real(64)
    st, nr, Q, _ = _refine(p)
    ref = oracle.refine(p.A, p.Qhat, lp="f32")
    assert st == B.SR_OK and nr.iters == ref.iters and nr.hp_gemms == 4 * nr.iters
    tol = oracle.default_tol(64)
    cT, cQ = oracle.residuals_dd(p.A, Q)
    assert cT <= tol and cQ <= tol
    assert np.max(np.abs(sign_align(Q, ref.Q) - ref.Q)) <= 1e-12
    assert np.max(np.abs(sign_align(Q, p.Q0) - p.Q0)) <= 1e-12


@pytest.mark.parametrize("n", [300, 1000])
def test_crt_refine_jittered(torch, n):
    p = inputs.jittered_real(n)
    st, nr, Q, _ = _refine(p)
    ref = oracle.refine(p.A, p.Qhat, lp="f32")
    assert st == B.SR_OK and abs(nr.iters - ref.iters) <= 1
    tol = oracle.default_tol(n)
    cT, cQ = oracle.residuals_dd(p.A, Q)
    assert cT <= tol and cQ <= tol
    Tq = np.diagonal(Q.T @ p.A @ Q)
    Tr = np.diagonal(ref.Q.T @ p.A @ ref.Q)
    assert np.max(np.abs(Tq - Tr)) <= 1e-12


def test_crt_one_pass_parity(torch):
    p = inputs.planted(96, inputs.eig_unit_step(96), 5, pert=1e-5)
    st, nr, Q, _ = _refine(p, max_iter=1)
    assert st == B.SR_ERR_NOT_CONVERGED and nr.iters == 1
    Q0, _ = oracle.ns_init(p.Qhat)
    Q1, info = oracle.iteration(p.A, Q0, lp="f32")
    assert nr.w_norm == pytest.approx(info.w_norm, rel=1e-5)
    assert np.max(np.abs(Q - Q1)) <= 50 * U32 * info.w_norm + 1e-13


def test_crt_refine_full_sigma_and_symmetric(torch):
    p = inputs.jittered_real(257)
    st, nr, Q, _ = _refine(p, full_sigma=1)
    ref = oracle.refine(p.A, p.Qhat, lp="f32", full_sigma=True)
    assert st == B.SR_OK and abs(nr.iters - ref.iters) <= 1
    tol = oracle.default_tol(257)
    cT, cQ = oracle.residuals_dd(p.A, Q)
    assert cT <= tol and cQ <= tol
    assert np.max(np.abs(sign_align(Q, ref.Q) - ref.Q)) <= 1e-9
    ps = inputs.symmetric_real(200)
    st, nr, Q, _ = _refine(ps, symmetric=1)
    ref = oracle.refine(ps.A, ps.Qhat, lp="f32", symmetric=True)
    assert st == B.SR_OK and abs(nr.iters - ref.iters) <= 1
    cT, cQ = oracle.residuals_dd(ps.A, Q)
    assert cT <= oracle.default_tol(200) and cQ <= oracle.default_tol(200)


@pytest.mark.parametrize("n", [96, 300])
def test_crt_complex_refine_matches_oracle(torch, n):
    p = inputs.ring_complex(n)
    st, nr, Q, T = _refine(p, cplx=True, T=True)
    ref = oracle.refine(p.A, p.Qhat, lp="f32")
    assert st == B.SR_OK and abs(nr.iters - ref.iters) <= 1
    tol = oracle.default_tol(n)
    cT, cQ = oracle.residuals_dd(p.A, Q)
    assert cT <= tol and cQ <= tol
    assert np.max(np.abs(phase_align(Q, ref.Q) - ref.Q)) <= 1e-11
    assert np.max(np.abs(np.diagonal(T) - p.lam)) <= 1e-12


def test_crt_headline_workload_full_size(torch):
    """The real n = 4096 workload with the residue form, as the benchmark runs
    it; sampled entries of Q^T A Q and Q^T Q - I recomputed by the oracle in
    double-double (see test_gpu_fullsize for the digit form)."""
    n = 4096
    p = inputs.jittered_real(n)
    st, nr, Q, T = _refine(p, T=True)
    tol = oracle.default_tol(n)
    assert st == B.SR_OK, B.status_string(st)
    assert nr.stril_rel <= tol and nr.orth <= np.sqrt(tol)
    rng = np.random.default_rng(4097)
    rows = np.concatenate([rng.integers(1, n, 96), np.arange(0, n, n // 16)])
    cols = np.concatenate([rng.integers(0, n - 1, 96), np.arange(0, n, n // 16)])
    rows, cols = np.maximum(rows, cols), np.minimum(rows, cols)
    t, y = oracle.sample_entries_dd(p.A, Q, rows, cols)
    anorm = np.linalg.norm(p.A)
    assert np.max(np.abs(T[rows, cols] - t)) <= 1e-13 * anorm
    low = rows > cols
    assert np.max(np.abs(t[low])) <= tol * anorm
    assert np.max(np.abs(y)) <= tol
    diag = rows == cols
    assert np.max(np.abs(t[diag] - p.lam[rows[diag]])) <= 1e-11


@pytest.mark.parametrize("n", [64, 512])
def test_crt_refine_nonnormal_unit_step(torch, n):
    """The unit-step spectrum with strictly upper entries of standard deviation
    1/sqrt(n) (the variance reading of "N(0, 1/n)"): strongly non-normal T0,
    against the oracle's refinement of the same input."""
    p = inputs.unit_step_real(n, upper_std=1.0 / np.sqrt(n))
    st, nr, Q, T = _refine(p, T=True)
    ref = oracle.refine(p.A, p.Qhat, lp="f32")
    assert st == B.SR_OK and ref.status == oracle.OK and abs(nr.iters - ref.iters) <= 1
    tol = oracle.default_tol(n)
    cT, cQ = oracle.residuals_dd(p.A, Q)
    assert cT <= tol and cQ <= tol
    # the Schur diagonal against the oracle's: eigenvalues of a non-normal T0 are
    # ill-conditioned (condition numbers kappa_i up to 5e7 at n = 64), so the two
    # may differ by about kappa_i u ||A|| (first-order perturbation by a backward
    # error of u ||A||): the bound is ten times that
    import scipy.linalg as sl
    w, VL, VR = sl.eig(p.T0, left=True, right=True)
    kappa = 1.0 / np.abs(np.sum(np.conj(VL) * VR, axis=0))
    order = np.argsort(w.real)
    kap = kappa[order]                       # the planted diagonal is ascending, like w
    Tr = ref.Q.T @ p.A @ ref.Q
    bound = 10 * kap * U64 * np.linalg.norm(p.A) + 1e-13
    assert np.all(np.abs(np.diagonal(T) - np.diagonal(Tr)) <= bound)
