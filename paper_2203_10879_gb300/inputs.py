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


def unit_step_real(n: int = 64, seed: int = BASE_SEED + 1, low: str = "f32") -> Planted:
    """Real planted problem with lambda_k = 1 + k/64 and a FP32-rounded start."""
    return planted(n, eig_unit_step(n), seed, pert=1e-6, low=low,
                   recipe=f"real n={n}, lambda_k=1+k/64, upper std 1/n, Qhat=fl_{low}(Q0 expm(1e-6 S))")


def jittered_real(n: int = 4096, seed: int = BASE_SEED + 2, low: str = "f32",
                  upper_std: float | None = None) -> Planted:
    """Real planted problem with lambda_k = k/n + U(0, 0.5/n)."""
    return planted(n, eig_jittered_grid(n, seed), seed, pert=1e-6, low=low, upper_std=upper_std,
                   recipe=f"real n={n}, lambda_k=k/n+U(0,0.5/n), upper std 1/n, Qhat=fl_{low}(Q0 expm(1e-6 S))")


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
