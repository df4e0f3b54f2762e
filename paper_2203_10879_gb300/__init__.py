"""GB300 (sm_103a) refinement of approximate Schur decompositions.

The Newton-like iteration of Bujanovic, Kressner and Schroeder (Alg. 4 of the
paper) runs in the CUDA library ``libschur_refine.so`` behind the C ABI in
``include/schur_refine.h``. This package holds its build script, the ctypes
binding (:mod:`._binding`, one function per C entry point) and the seeded input
generators (:mod:`.inputs`). Importing the package does not load the library;
the first binding call does, and fails loudly if it is missing.
"""
from . import _binding as binding  # noqa: F401
from ._binding import (  # noqa: F401
    SchurRefineError, default_options, colmajor, status_string,
    schur_refine_create, schur_refine_step, schur_refine_batched, schur_refine_residuals,
    schur_refine_trisolve, schur_refine_gemm, schur_refine_get_profile, schur_refine_reset_profile,
    schur_refine_destroy,
)


class Refiner:
    """Owns one library handle; every method is one C call.

    ``Refiner(n_max, **options)``; options are the fields of ``sr_options``
    (dtype, hp_gemm, lp, qhat_type, full_sigma, max_iter, ozaki_slices, tol,
    profile). Tensors are CUDA, column-major.
    """

    def __init__(self, n_max: int, stream=None, **options):
        import torch
        self.n_max = int(n_max)
        self.opt = default_options(**options)
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        s, self.h = schur_refine_create(self.n_max, self.opt, stream)
        if s != 0:
            raise SchurRefineError(s, "schur_refine_create")

    def step(self, A, Q, Qhat=None, T=None, check=True):
        s, nr = schur_refine_step(self.h, A.shape[0], A, Q, Qhat, T)
        if check and s not in (0,):
            raise SchurRefineError(s, "schur_refine_step")
        return s, nr

    def residuals(self, A, Q):
        s, a, b = schur_refine_residuals(self.h, A.shape[0], A, Q)
        if s != 0:
            raise SchurRefineError(s, "schur_refine_residuals")
        return a, b

    def profile(self) -> dict:
        s, p = schur_refine_get_profile(self.h)
        if s != 0:
            raise SchurRefineError(s, "schur_refine_get_profile")
        return p.as_dict()

    def reset_profile(self):
        schur_refine_reset_profile(self.h)

    def close(self):
        if getattr(self, "h", None):
            schur_refine_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
