"""GB300-native FEAST contour-filter eigensolver (real symmetric and complex Hermitian
sparse problems).

Thin Python binding over the C ABI of ``libfeast_gb300.so`` (declared in
``include/feast_gb300.h``).  Every step of the method runs in the library's
CUDA kernels; this module only marshals arguments: numpy arrays for the host
entry points, torch CUDA tensors (device memory, current stream) for the
device entry points.  There is no CPU fallback: if the library is missing or
no GPU is present the calls raise.
"""
from __future__ import annotations

from ._lib import (  # noqa: F401
    FeastError,
    FeastResult,
    feast_contour_nodes,
    feast_contour_nodes_rule,
    feast_eig_grad_dev,
    feast_filter_dev,
    feast_filter_layout,
    feast_gemm_dev,
    feast_gemm_oz_dev,
    feast_gram_dev,
    feast_gram_noalloc_dev,
    feast_gram_oz_dev,
    feast_hcsr_solve,
    feast_hcsr_solve_dev,
    feast_hcsr_workspace_bytes,
    feast_init,
    feast_last_error,
    feast_last_profile,
    feast_reduced_eig_dev,
    feast_residual_dev,
    feast_scsr_solve,
    feast_scsr_solve_batched,
    feast_scsr_solve_dev,
    feast_scsr_solve_dev_x,
    feast_scsr_solve_x,
    feast_scsr_extreme,
    feast_scsr_extreme_dev,
    feast_scsr_grad,
    feast_scsr_workspace_bytes,
    feast_set_wait_limit,
    feast_shifted_spmm_dev,
    feast_sym_eig_dev,
    library,
    library_path,
)

__all__ = [n for n in dir() if n.startswith("feast_")] + ["FeastError", "FeastResult", "library",
                                                          "library_path"]
