"""Seeded synthetic inputs: planted approximate Schur decompositions.

This module builds test and benchmark inputs only. It holds none of the
refinement method's arithmetic (no residual, no triangular solve, no
Newton-Schulz step); both the CUDA path and the CPU oracle consume the arrays it
returns.

Every input follows the problem statement of Sec. 2 (eq. (2.1), "lowup"): a
matrix ``A`` and a nearly unitary ``Qhat`` for which ``Qhat^H A Qhat`` is nearly
upper triangular. The decomposition is planted: ``A = Q0 T0 Q0^H`` with ``T0``
upper triangular (distinct diagonal, as Theorem 1 requires), and ``Qhat`` is
``Q0 expm(eps S)`` with ``S`` skew-Hermitian, rounded to the low precision.

Random numbers come from a counter-based SplitMix64 generator (Steele, Lea,
Flood 2014) and Box-Muller normals, written out here so that a given seed yields
the same stream on every machine and numpy version.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

#: Seed base for the named workloads; workload k uses BASE_SEED + k.
BASE_SEED = 2203108790


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs ``start .. start+count-1`` of the SplitMix64 stream for ``seed``."""
    with np.errstate(over="ignore"):
        idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


class Stream:
    """Sequential view of a counter-based SplitMix64 stream."""

    def __init__(self, seed: int):
        self.seed = int(seed)
        self.pos = 0

    def bits(self, count: int) -> np.ndarray:
        out = splitmix64(self.seed, self.pos, count)
        self.pos += count
        return out

    def uniform(self, shape) -> np.ndarray:
        """Uniform on the open interval (0, 1), 53 random bits each."""
        count = int(np.prod(shape))
        b = self.bits(count)
        u = ((b >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)
        return u.reshape(shape)

    def normal(self, shape) -> np.ndarray:
        """Standard normals by the Box-Muller transform."""
        count = int(np.prod(shape))
        half = (count + 1) // 2
        u1 = self.uniform((half,))
        u2 = self.uniform((half,))
        r = np.sqrt(-2.0 * np.log(u1))
        z = np.concatenate([r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2)])
        return z[:count].reshape(shape)


def _haar_orthogonal(st: Stream, n: int, complex_: bool) -> np.ndarray:
    """Q factor of a seeded Gaussian matrix, signs fixed so diag(R) > 0."""
    g = st.normal((n, n))
    if complex_:
        g = (g + 1j * st.normal((n, n))) / math.sqrt(2.0)
    q, r = np.linalg.qr(g)
    d = np.diagonal(r)
    ph = d / np.abs(d)
    return np.asfortranarray(q * ph[None, :])


def _skew(st: Stream, n: int, complex_: bool) -> np.ndarray:
    """Skew-Hermitian S: iid N(0,1) strictly-lower entries mirrored with a minus sign.

    In the complex case the strictly-lower entries are complex N(0,1) and the
    diagonal is i*N(0,1).
    """
    g = st.normal((n, n))
    if complex_:
        g = g + 1j * st.normal((n, n))
    low = np.tril(g, -1)
    s = low - low.conj().T
    if complex_:
        s = s + 1j * np.diag(st.normal((n,)))
    return s


def _expm_small(x: np.ndarray, degree: int) -> np.ndarray:
    """Taylor polynomial of exp(x); for ||x|| <~ 1e-2 the omitted terms are far below 1e-16."""
    n = x.shape[0]
    term = x.copy()                       # the k = 1 term, I x / 1, without a product
    out = np.eye(n, dtype=x.dtype) + term
    for k in range(2, degree + 1):
        term = term @ x / k
        out = out + term
    return out


@dataclass
class Planted:
    """A planted decomposition A = Q0 T0 Q0^H with its perturbed starting factor."""

    A: np.ndarray          # n x n, float64 or complex128, Fortran order
    Qhat: np.ndarray       # n x n, low precision (float32 / complex64 / float64)
    Q0: np.ndarray         # exact factor the perturbation was applied to
    T0: np.ndarray         # planted upper triangular factor
    lam: np.ndarray        # planted eigenvalues, diag(T0)
    seed: int
    recipe: str

    @property
    def n(self) -> int:
        return self.A.shape[0]


def _cache_path(key: str) -> str | None:
    """File under $SR_INPUT_CACHE for a generated input (no caching when unset)."""
    import hashlib
    import os
    d = os.environ.get("SR_INPUT_CACHE")
    if not d:
        return None
    os.makedirs(d, exist_ok=True)
    return os.path.join(d, hashlib.sha256(key.encode()).hexdigest()[:32] + ".npz")


def planted(n: int, lam: np.ndarray, seed: int, *, pert: float = 1e-6,
            low: str = "f32", complex_: bool = False, recipe: str = "",
            upper_std: float | None = None) -> Planted:
    """Build A = Q0 T0 Q0^H and Qhat = fl_low(Q0 expm(pert*S)); see _planted.

    With the environment variable SR_INPUT_CACHE set to a directory, the arrays
    are kept there and read back by later calls with the same arguments (large
    orders take minutes of host BLAS to build)."""
    lam = np.asarray(lam)
    path = _cache_path(repr((n, hashlib_digest(lam), seed, pert, low, complex_, upper_std)))
    if path is not None:
        import os
        if os.path.exists(path):
            z = np.load(path)
            return Planted(A=np.asfortranarray(z["A"]), Qhat=np.asfortranarray(z["Qhat"]),
                           Q0=np.asfortranarray(z["Q0"]), T0=np.asfortranarray(z["T0"]), lam=z["lam"],
                           seed=seed, recipe=recipe)
    p = _planted(n, lam, seed, pert=pert, low=low, complex_=complex_, recipe=recipe, upper_std=upper_std)
    if path is not None:
        tmp = path + ".tmp.npz"
        np.savez(tmp, A=p.A, Qhat=p.Qhat, Q0=p.Q0, T0=p.T0, lam=p.lam)
        import os
        os.replace(tmp, path)
    return p


def hashlib_digest(a: np.ndarray) -> str:
    import hashlib
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def _planted(n: int, lam: np.ndarray, seed: int, *, pert: float = 1e-6,
             low: str = "f32", complex_: bool = False, recipe: str = "",
             upper_std: float | None = None) -> Planted:
    """Build A = Q0 T0 Q0^H and Qhat = fl_low(Q0 expm(pert*S)).

    T0 has diagonal ``lam`` and iid normal strictly-upper entries with mean 0
    and standard deviation ``upper_std`` (default 1/n). In the complex case the
    entries are complex normal with that standard deviation (real and imaginary
    parts each upper_std/sqrt(2)).

    With standard deviation 1/sqrt(n) instead, a spectrum packed at spacing
    ~1/n makes the triangular equation so ill-conditioned that the iteration
    diverges from an FP32 start; that variant serves as a failure-path input.
    """
    st = Stream(seed)
    lam = np.asarray(lam)
    sd = (1.0 / n) if upper_std is None else float(upper_std)
    up = st.normal((n, n)) * sd
    if complex_:
        up = (up + 1j * st.normal((n, n)) * sd) / math.sqrt(2.0)
    T0 = np.triu(up, 1) + np.diag(lam.astype(np.complex128 if complex_ else np.float64))
    Q0 = _haar_orthogonal(st, n, complex_)
    A = np.asfortranarray((Q0 @ T0) @ Q0.conj().T)
    S = _skew(st, n, complex_)
    P = _expm_small(pert * S, 6)
    Qexact = Q0 @ P
    dt = {"f32": np.complex64 if complex_ else np.float32,
          "f64": np.complex128 if complex_ else np.float64}[low]
    Qhat = np.asfortranarray(Qexact.astype(dt))
    return Planted(A=A, Qhat=Qhat, Q0=Q0, T0=np.asfortranarray(T0), lam=lam,
                   seed=seed, recipe=recipe)


def eig_unit_step(n: int) -> np.ndarray:
    """lambda_k = 1 + k/64, k = 0..n-1 (distinct, gap 1/64)."""
    return 1.0 + np.arange(n, dtype=np.float64) / 64.0


def eig_jittered_grid(n: int, seed: int) -> np.ndarray:
    """lambda_k = k/n + U(0, 0.5/n), sorted; consecutive gaps lie in (0.5/n, 1.5/n)."""
    st = Stream(seed ^ 0x5EED)
    lam = np.arange(n, dtype=np.float64) / n + st.uniform((n,)) * (0.5 / n)
    return np.sort(lam)


def eig_ring(n: int, seed: int) -> np.ndarray:
    """0.5 exp(2 pi i k/n)(1 + U(0, 0.2)): distinct complex eigenvalues on a ring."""
    st = Stream(seed ^ 0x5EED)
    k = np.arange(n, dtype=np.float64)
    return 0.5 * np.exp(2j * np.pi * k / n) * (1.0 + 0.2 * st.uniform((n,)))


def unit_step_real(n: int = 64, seed: int = BASE_SEED + 1, low: str = "f32",
                   upper_std: float | None = None) -> Planted:
    """Real planted problem with lambda_k = 1 + k/64 and a FP32-rounded start.

    The strictly upper entries of T0 have standard deviation 1/n unless
    upper_std is given (1/sqrt(n) is the variance-1/n reading of "N(0, 1/n)")."""
    sd = 1.0 / n if upper_std is None else float(upper_std)
    return planted(n, eig_unit_step(n), seed, pert=1e-6, low=low, upper_std=sd,
                   recipe=f"real n={n}, lambda_k=1+k/64, upper std {sd:.3g}, Qhat=fl_{low}(Q0 expm(1e-6 S))")


def jittered_real(n: int = 4096, seed: int = BASE_SEED + 2, low: str = "f32",
                  upper_std: float | None = None) -> Planted:
    """Real planted problem with lambda_k = k/n + U(0, 0.5/n)."""
    return planted(n, eig_jittered_grid(n, seed), seed, pert=1e-6, low=low, upper_std=upper_std,
                   recipe=f"real n={n}, lambda_k=k/n+U(0,0.5/n), upper std 1/n, Qhat=fl_{low}(Q0 expm(1e-6 S))")


def symmetric_real(n: int = 4096, seed: int = BASE_SEED + 5, low: str = "f32") -> Planted:
    """Real symmetric planted problem (Sec. 2.5): T0 = diag(lambda), lambda_k =
    k/n + U(0, 0.5/n); A = Q0 T0 Q0^T made exactly symmetric, (A + A^T)/2."""
    p = planted(n, eig_jittered_grid(n, seed), seed, pert=1e-6, low=low, upper_std=0.0,
                recipe=f"real symmetric n={n}, A=Q0 diag(lambda) Q0^T, lambda_k=k/n+U(0,0.5/n), "
                       f"Qhat=fl_{low}(Q0 expm(1e-6 S))")
    A = np.asfortranarray(0.5 * (p.A + p.A.T))
    return Planted(A=A, Qhat=p.Qhat, Q0=p.Q0, T0=p.T0, lam=p.lam, seed=p.seed, recipe=p.recipe)


def quasi_real(n: int = 4096, seed: int = BASE_SEED + 8, pair_prob: float = 1.0 / 3.0,
               low: str = "f32") -> Planted:
    """Real planted problem whose Schur form is quasi-triangular (Sec. 3: real
    Schur decompositions, 2 x 2 diagonal blocks for complex-conjugate pairs).

    Base values mu_k = k/n + U(0, 0.5/n) (sorted, as the jittered grid). Going
    down the diagonal, a 2 x 2 block starts at row k (k + 1 < n) with
    probability pair_prob; it is [[alpha, beta s], [-beta/s, alpha]] with
    alpha = (mu_k + mu_k+1)/2, beta = (mu_k+1 - mu_k) U(0.5, 1.5), s = 2^U(-1, 1),
    eigenvalues alpha +- i beta; other rows are 1 x 1 blocks mu_k. Entries above
    the blocks: normal with standard deviation 1/n. A = Q0 T0 Q0^T in FP64,
    Qhat = fl_low(Q0 expm(1e-6 S)). `lam` holds the planted eigenvalues row by
    row (alpha + i beta, alpha - i beta for a block) and `blk` the block sizes
    (2 at a block's first row, 0 at its second, else 1)."""
    st = Stream(seed)
    mu = np.sort(np.arange(n, dtype=np.float64) / n + st.uniform((n,)) * (0.5 / n))
    u = st.uniform((n, 3))
    blk = np.ones(n, dtype=np.int32)
    T0 = np.triu(st.normal((n, n)) * (1.0 / n), 1)
    lam = mu.astype(np.complex128)
    k = 0
    while k < n:
        if k + 1 < n and u[k, 0] < pair_prob:
            alpha = 0.5 * (mu[k] + mu[k + 1])
            beta = (mu[k + 1] - mu[k]) * (0.5 + u[k, 1])
            sc = 2.0 ** (2.0 * u[k, 2] - 1.0)
            T0[k, k] = T0[k + 1, k + 1] = alpha
            T0[k, k + 1] = beta * sc
            T0[k + 1, k] = -beta / sc
            lam[k], lam[k + 1] = alpha + 1j * beta, alpha - 1j * beta
            blk[k], blk[k + 1] = 2, 0
            k += 2
        else:
            T0[k, k] = mu[k]
            k += 1
    Q0 = _haar_orthogonal(st, n, False)
    A = np.asfortranarray((Q0 @ T0) @ Q0.T)
    S = _skew(st, n, False)
    Qhat = np.asfortranarray((Q0 @ _expm_small(1e-6 * S, 6)).astype(np.float32 if low == "f32" else np.float64))
    p = Planted(A=A, Qhat=Qhat, Q0=Q0, T0=np.asfortranarray(T0), lam=lam, seed=seed,
                recipe=f"real quasi-triangular n={n}, pairs with probability {pair_prob:.3g}, "
                       f"Qhat=fl_{low}(Q0 expm(1e-6 S))")
    p.blk = blk
    return p


def hermitian_complex(n: int = 2048, seed: int = BASE_SEED + 7, low: str = "f32") -> Planted:
    """Complex Hermitian planted problem (Sec. 2.5): T0 = diag(lambda) real,
    lambda_k = k/n + U(0, 0.5/n); A = Q0 T0 Q0^H with Q0 Haar unitary, made
    exactly Hermitian, (A + A^H)/2; Qhat = fl_c64(Q0 expm(1e-6 S)), S
    skew-Hermitian."""
    p = planted(n, eig_jittered_grid(n, seed), seed, pert=1e-6, low=low, complex_=True, upper_std=0.0,
                recipe=f"complex Hermitian n={n}, A=Q0 diag(lambda) Q0^H, lambda_k=k/n+U(0,0.5/n), "
                       f"Qhat=fl_c64(Q0 expm(1e-6 S))")
    A = np.asfortranarray(0.5 * (p.A + p.A.conj().T))
    return Planted(A=A, Qhat=p.Qhat, Q0=p.Q0, T0=p.T0, lam=p.lam, seed=p.seed, recipe=p.recipe)


def clustered_complex(n: int = 150, cond: float = 1e5, radius: float = 1e-5, seed: int = BASE_SEED + 6,
                      low: str = "f32") -> Planted:
    """The setting of Example 3 (Sec. 3): A = X D X^-1 with X of condition
    ``cond`` (singular values geometric between 1 and 1/cond, Haar singular
    vectors) and D real diagonal, uniform in [-10, 10] except two clusters of
    10 eigenvalues within ``radius`` of random centres. The start is the
    complex Schur form computed by LAPACK in FP64 (scipy.linalg.schur), the
    Schur vectors rounded to ``low``; Q0 holds the FP64 Schur vectors and T0
    the FP64 Schur factor."""
    import scipy.linalg
    st = Stream(seed)
    U = _haar_orthogonal(st, n, False)
    V = _haar_orthogonal(st, n, False)
    sv = np.exp(-np.log(cond) * np.arange(n) / (n - 1))
    X = (U * sv) @ V.T
    lam = -10.0 + 20.0 * st.uniform((n,))
    for c in range(2):
        centre = -10.0 + 20.0 * float(st.uniform((1,))[0])
        lam[10 * c:10 * c + 10] = centre + radius * (2.0 * st.uniform((10,)) - 1.0)
    A = np.asfortranarray(np.linalg.solve(X.T, (X * lam).T).T)   # X diag(lam) X^-1
    Ac = A.astype(np.complex128)
    T0, Z = scipy.linalg.schur(Ac, output="complex")
    dt = {"f32": np.complex64, "f64": np.complex128}[low]
    return Planted(A=np.asfortranarray(Ac), Qhat=np.asfortranarray(Z.astype(dt)), Q0=np.asfortranarray(Z),
                   T0=np.asfortranarray(T0), lam=lam, seed=seed,
                   recipe=f"Example 3 setting n={n}: A = X D X^-1, cond(X)={cond:g}, two clusters of 10 within "
                          f"{radius:g}; Qhat = fl_{low}(complex Schur vectors of LAPACK in FP64)")


def ring_complex(n: int = 8192, seed: int = BASE_SEED + 3) -> Planted:
    """Complex planted problem with ring eigenvalues and a complex64-rounded start."""
    return planted(n, eig_ring(n, seed), seed, pert=1e-6, low="f32", complex_=True,
                   recipe=f"complex n={n}, ring eigenvalues, complex upper std 1/n, Qhat=fl_c64(Q0 expm(1e-6 S))")


def batch_sizes(count: int = 1024, lo: int = 32, hi: int = 512, seed: int = BASE_SEED + 4) -> np.ndarray:
    """n = round(exp(U(ln lo, ln hi))) for each of ``count`` matrices."""
    st = Stream(seed)
    u = st.uniform((count,))
    return np.rint(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)


def batch_problem(i: int, n: int, seed: int = BASE_SEED + 4) -> Planted:
    """Matrix ``i`` of the batched workload, built like the unit-step real problem."""
    return unit_step_real(int(n), seed=seed * 4099 + i + 1, low="f32")


# ---------------------------------------------------------------------------
# Double-double planted problems (working precision above FP64)
#
# A pair of float64 arrays (hi, lo) stands for the unevaluated sum hi + lo.
# The factor Q0 is built from rotations whose cosine and sine are exact
# rationals, so that Q0 is orthogonal to double-double accuracy without any
# orthogonalisation step: two butterfly networks (stage b rotates the rows i
# and i + 2^b for every i with bit b clear) around a random row permutation.
# Applying the rotations to T0 from both sides gives A = Q0 T0 Q0^T in
# double-double with a few roundings per entry. The elementary operations are
# the error-free transformations of Knuth (TwoSum) and Dekker (Veltkamp
# splitting, TwoProduct), written out for numpy arrays (no fused multiply-add
# is assumed).

_SPLITTER = 134217729.0   # 2^27 + 1


def _two_sum(a, b):
    s = a + b
    bb = s - a
    return s, (a - (s - bb)) + (b - bb)


def _quick_two_sum(a, b):
    s = a + b
    return s, b - (s - a)


def _split(a):
    t = _SPLITTER * a
    hi = t - (t - a)
    return hi, a - hi


def _two_prod(a, b):
    p = a * b
    ah, al = _split(a)
    bh, bl = _split(b)
    return p, ((ah * bh - p) + ah * bl + al * bh) + al * bl


def _dd_add(ah, al, bh, bl):
    s, e = _two_sum(ah, bh)
    t, f = _two_sum(al, bl)
    s, e = _quick_two_sum(s, e + t)
    return _quick_two_sum(s, e + f)


def _dd_mul(ah, al, bh, bl):
    p, e = _two_prod(ah, bh)
    return _quick_two_sum(p, e + (ah * bl + al * bh))


def _dd_div(nh, d):
    """(nh / d) in double-double for float64 nh, d."""
    q = nh / d
    p, e = _two_prod(q, d)
    r = (nh - p) - e
    return _quick_two_sum(q, r / d)


def _rotation_set(st: Stream, count: int):
    """cos/sin pairs c = (1 - t^2)/(1 + t^2), s = 2t/(1 + t^2) in double-double,
    t = k / 2^20 with k uniform in [-2^20, 2^20]: numerators and denominator are
    exact in float64, so c^2 + s^2 = 1 up to the double-double rounding."""
    k = np.floor(st.uniform((count,)) * (2.0 ** 21 + 1.0)) - 2.0 ** 20
    t = k * 2.0 ** -20
    t2 = t * t                                 # exact: k^2 < 2^41
    den = 1.0 + t2
    ch, cl = _dd_div(1.0 - t2, den)
    sh, sl = _dd_div(2.0 * t, den)
    return ch, cl, sh, sl


@dataclass
class _Butterflies:
    n: int
    stages: list          # per stage: (rows i, rows i + 2^b, c_hi, c_lo, s_hi, s_lo)
    perm: np.ndarray      # row permutation between the two networks
    split: int            # stages before the permutation


def _make_butterflies(st: Stream, n: int) -> _Butterflies:
    nb = max(1, int(math.ceil(math.log2(max(n, 2)))))
    stages = []
    for _ in range(2):
        for b in range(nb):
            i = np.arange(n)
            i = i[((i >> b) & 1) == 0]
            i = i[i + (1 << b) < n]
            stages.append((i, i + (1 << b)) + _rotation_set(st, len(i)))
    perm = np.argsort(st.uniform((n,)), kind="stable")
    return _Butterflies(n=n, stages=stages, perm=perm, split=nb)


def _apply_rows(bf: _Butterflies, Xh: np.ndarray, Xl: np.ndarray):
    """(Xh, Xl) <- Q0 (Xh, Xl): the rotations applied to the rows, in double-double."""
    Xh = Xh.copy()
    Xl = Xl.copy()
    for k, (i, j, ch, cl, sh, sl) in enumerate(bf.stages):
        if k == bf.split:
            Xh = Xh[bf.perm]
            Xl = Xl[bf.perm]
        ch, cl, sh, sl = (v[:, None] for v in (ch, cl, sh, sl))
        xh, xl, yh, yl = Xh[i], Xl[i], Xh[j], Xl[j]
        p1 = _dd_mul(ch, cl, xh, xl)
        p2 = _dd_mul(sh, sl, yh, yl)
        p3 = _dd_mul(sh, sl, xh, xl)
        p4 = _dd_mul(ch, cl, yh, yl)
        Xh[i], Xl[i] = _dd_add(p1[0], p1[1], -p2[0], -p2[1])     # c x - s y
        Xh[j], Xl[j] = _dd_add(p3[0], p3[1], p4[0], p4[1])       # s x + c y
    return Xh, Xl


@dataclass
class PlantedDD:
    """A = Q0 T0 Q0^T held as double-double planes, with a float64 start."""

    A_hi: np.ndarray
    A_lo: np.ndarray
    Qhat: np.ndarray       # float64 starting factor
    Q0_hi: np.ndarray
    Q0_lo: np.ndarray
    T0: np.ndarray         # float64, upper triangular
    lam: np.ndarray
    seed: int
    recipe: str

    @property
    def n(self) -> int:
        return self.A_hi.shape[0]


def planted_dd(n: int, lam: np.ndarray, seed: int, *, pert: float = 1e-14,
               recipe: str = "", upper_std: float | None = None) -> PlantedDD:
    """A = Q0 T0 Q0^T in double-double, Qhat = fl64(Q0 expm(pert S)).

    T0 has diagonal ``lam`` and iid normal strictly-upper entries with standard
    deviation ``upper_std`` (default 1/n; float64, exact in double-double). Q0
    is the butterfly factor described above. Cached under $SR_INPUT_CACHE like
    :func:`planted`."""
    lam = np.asarray(lam, dtype=np.float64)
    key = ("dd", n, hashlib_digest(lam), seed, pert) + (() if upper_std is None else (upper_std,))
    path = _cache_path(repr(key))
    if path is not None:
        import os
        if os.path.exists(path):
            z = np.load(path)
            f = lambda k: np.asfortranarray(z[k])
            return PlantedDD(A_hi=f("A_hi"), A_lo=f("A_lo"), Qhat=f("Qhat"), Q0_hi=f("Q0_hi"),
                             Q0_lo=f("Q0_lo"), T0=f("T0"), lam=z["lam"], seed=seed, recipe=recipe)
    st = Stream(seed)
    sd = (1.0 / n) if upper_std is None else float(upper_std)
    T0 = np.triu(st.normal((n, n)) * sd, 1) + np.diag(lam)
    bf = _make_butterflies(st, n)
    z = np.zeros((n, n))
    Q0h, Q0l = _apply_rows(bf, np.eye(n), z)
    Mh, Ml = _apply_rows(bf, T0, z)                   # Q0 T0
    Ah, Al = _apply_rows(bf, Mh.T, Ml.T)              # Q0 (Q0 T0)^T = (Q0 T0 Q0^T)^T
    Ah, Al = Ah.T, Al.T
    # Qhat = fl64(Q0 + Q0 (expm(pert S) - I)); the correction is ~pert*n, so
    # float64 products give it far below the final rounding
    S = _skew(st, n, False)
    X = pert * S
    D = X + X @ X / 2.0 + X @ X @ X / 6.0             # expm(X) - I to third order
    C = Q0h @ D
    qh, ql = _dd_add(Q0h, Q0l, C, np.zeros_like(C))
    Qhat = qh + ql
    p = PlantedDD(A_hi=np.asfortranarray(Ah), A_lo=np.asfortranarray(Al), Qhat=np.asfortranarray(Qhat),
                  Q0_hi=np.asfortranarray(Q0h), Q0_lo=np.asfortranarray(Q0l), T0=np.asfortranarray(T0),
                  lam=lam, seed=seed, recipe=recipe)
    if path is not None:
        import os
        tmp = path + ".tmp.npz"
        np.savez(tmp, A_hi=p.A_hi, A_lo=p.A_lo, Qhat=p.Qhat, Q0_hi=p.Q0_hi, Q0_lo=p.Q0_lo, T0=p.T0, lam=p.lam)
        os.replace(tmp, path)
    return p


def unit_step_dd(n: int = 2048, seed: int = BASE_SEED + 5, upper_std: float | None = None) -> PlantedDD:
    """Double-double planted problem, lambda_k = 1 + k/64, Qhat = fl64(Q0 expm(1e-14 S));
    strictly upper entries of standard deviation 1/n unless upper_std is given."""
    sd = 1.0 / n if upper_std is None else float(upper_std)
    return planted_dd(n, eig_unit_step(n), seed, pert=1e-14, upper_std=sd,
                      recipe=f"real n={n} double-double, lambda_k=1+k/64, upper std {sd:.3g}, "
                             f"Qhat=fl64(Q0 expm(1e-14 S))")


# ---------------------------------------------------------------------------
# Planted problems whose Schur decomposition is known exactly (working
# precisions above double-double)
#
# For n a power of two, Q0 = D1 P1 (H D2 H / n) P2, with H the Sylvester
# Hadamard matrix (entries +-1, H H = n I), D1, D2 random sign diagonals and
# P1, P2 random permutations, is exactly orthogonal, and its entries are
# multiples of 1/n. With T0 upper triangular of dyadic entries (multiples of
# 2^-20), every entry of Q0 T0 and of (Q0 T0) Q0^T, and every partial sum of
# the float64 products that form them, is a multiple of 2^-20 / n^2 below
# ||T0||_2 in magnitude (Cauchy-Schwarz over any subset of the terms): below
# 2^53 units while ||T0||_2 < 2^53 / (2^20 n^2), so float64 forms
# A = Q0 T0 Q0^T exactly. The refined factors can then be compared with the
# exact Q0 and T0 at any precision.

@dataclass
class PlantedExact:
    """A = Q0 T0 Q0^T exactly in float64, Q0 exactly orthogonal, float64 start."""

    A: np.ndarray
    Qhat: np.ndarray
    Q0: np.ndarray
    T0: np.ndarray
    lam: np.ndarray
    seed: int
    recipe: str

    @property
    def n(self) -> int:
        return self.A.shape[0]


def _sylvester_hadamard(n: int) -> np.ndarray:
    H = np.ones((1, 1))
    while H.shape[0] < n:
        H = np.block([[H, H], [H, -H]])
    return H


def planted_exact(n: int, lam: np.ndarray, seed: int, *, pert: float = 1e-14, upper_std: float | None = None,
                  frac_bits: int = 20, recipe: str = "") -> PlantedExact:
    """The exact planted problem described above. ``lam`` must be dyadic (it is
    the diagonal of T0 as given); the strictly upper entries are normal with
    standard deviation ``upper_std`` (default 1/n) rounded to multiples of
    2^-frac_bits. Qhat = fl64(Q0 expm(pert S)), S skew-symmetric N(0,1)."""
    if n < 1 or n & (n - 1):
        raise ValueError("n must be a power of two")
    lam = np.asarray(lam, dtype=np.float64)
    st = Stream(seed)
    sd = (1.0 / n) if upper_std is None else float(upper_std)
    scale = float(2 ** frac_bits)
    U = np.round(st.normal((n, n)) * sd * scale) / scale
    T0 = np.triu(U, 1) + np.diag(lam)
    H = _sylvester_hadamard(n)
    d1 = np.where(st.uniform((n,)) < 0.5, -1.0, 1.0)
    d2 = np.where(st.uniform((n,)) < 0.5, -1.0, 1.0)
    p1 = np.argsort(st.uniform((n,)), kind="stable")
    p2 = np.argsort(st.uniform((n,)), kind="stable")
    C = (H * d2[None, :]) @ H / n                       # H D2 H / n, exact
    Q0 = np.asfortranarray(d1[:, None] * C[p1][:, p2])
    A = np.asfortranarray((Q0 @ T0) @ Q0.T)
    S = _skew(st, n, False)
    X = pert * S
    D = X + X @ X / 2.0 + X @ X @ X / 6.0               # expm(X) - I to third order
    Qhat = np.asfortranarray(Q0 + Q0 @ D)
    return PlantedExact(A=A, Qhat=Qhat, Q0=Q0, T0=np.asfortranarray(T0), lam=lam, seed=seed,
                        recipe=recipe or f"real n={n} exact planted (Hadamard Q0), upper std {sd:.3g} "
                                         f"in multiples of 2^-{frac_bits}, Qhat=fl64(Q0 expm({pert:g} S))")


def unit_step_exact(n: int = 2048, seed: int = BASE_SEED + 9) -> PlantedExact:
    """The triple-double workload: lambda_k = 1 + k/64 (dyadic), exact A."""
    return planted_exact(n, eig_unit_step(n), seed, pert=1e-14,
                         recipe=f"real n={n} exact planted A=Q0 T0 Q0^T (Q0 = D1 P1 H D2 H P2 / n, Hadamard H), "
                                f"lambda_k=1+k/64, upper std 1/n in multiples of 2^-20, "
                                f"Qhat=fl64(Q0 expm(1e-14 S))")
