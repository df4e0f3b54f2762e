"""CPU oracle for the Schur refinement iteration -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. It shares no code with the CUDA library
and never calls it. See :mod:`oracle.alg` for what each function follows;
:mod:`oracle.ddtarget` holds the double-double working-precision form of Alg. 4,
:mod:`oracle.mptarget` the form with an exact fixed-point high precision that
checks the multi-word (triple-double) forms.
"""
from ._lib import build, set_threads, max_threads  # noqa: F401
from .alg import (  # noqa: F401
    OK, NONDISTINCT, NONFINITE, NOT_CONVERGED, SolveError, IterInfo, RefineResult,
    alg2, sym_solve, alg3, kron_solve, ns_init, form_residual, iteration, refine, default_tol,
    quasi_blocks, block_lower_mask, alg2_quasi,
    residuals_dd, sample_entries_dd, gemm_dd,
)
