"""Helpers shared by the GPU tests: moving column-major matrices to and from the device."""
import numpy as np


def to_dev(a: np.ndarray):
    """A CUDA tensor with column-major layout holding the numpy matrix ``a``."""
    import torch
    a = np.asarray(a)
    if a.ndim == 1:
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return torch.from_numpy(np.ascontiguousarray(a.T)).cuda().t()


def from_dev(t) -> np.ndarray:
    if t.dim() == 1:
        return t.cpu().numpy()
    return np.asfortranarray(t.t().contiguous().cpu().numpy().T)


def empty_dev(n: int, m: int, dtype):
    import torch
    return torch.empty((m, n), dtype=dtype, device="cuda").t()


def sign_align(Q: np.ndarray, R: np.ndarray) -> np.ndarray:
    """Q with each column's sign flipped to match R (real case)."""
    s = np.sign(np.sum(Q * R, axis=0))
    s[s == 0] = 1.0
    return Q * s


def phase_align(Q: np.ndarray, R: np.ndarray) -> np.ndarray:
    """Q with each column multiplied by the unit-modulus factor that best matches R."""
    c = np.sum(np.conj(Q) * R, axis=0)
    a = np.abs(c)
    ph = np.where(a > 0, c / np.where(a > 0, a, 1.0), 1.0)
    return Q * ph
