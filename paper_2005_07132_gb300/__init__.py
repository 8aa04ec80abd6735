"""GB300-native fKK-EC (factorised Kramers-Kronig with phase- and scale-error
correction, arXiv 2005.07132).

The compute lives in libfkk.so (C ABI: include/fkk.h), hand-written CUDA for
sm_103a; this package is its thin Python binding (`_lib`), the in-tree build
(`build`) and the seeded synthetic input generator (`synth`).  Importing the
package does not load the library; the first binding call does, and raises
if the library has not been built.
"""
from ._lib import (  # noqa: F401
    PREC_BF16,
    PREC_BF16X3,
    SEC_MEAN,
    SEC_SAVGOL,
    SVD_EXACT,
    SVD_RANDOMIZED,
    Basis,
    Context,
    FitParams,
    FkkError,
    fit_params,
    fkk_apply,
    fkk_basis_from_arrays,
    fkk_basis_load,
    fkk_basis_math,
    fkk_eig_topk,
    fkk_refine_basis,
    fkk_fit_basis,
    fkk_fit_many,
    CubeJob,
    fkk_gram,
    fkk_noise_scale,
    fkk_project,
    fkk_reconstruct,
    fkk_reconstruct_noalloc,
    kk_per_spectrum,
    conventional_per_spectrum,
    fkk_residual,
    fkk_philox_normals,
    launch_count,
    lib,
    Server,
)

__all__ = [
    "Basis", "Context", "FitParams", "FkkError", "PREC_BF16", "PREC_BF16X3", "SEC_MEAN", "SEC_SAVGOL", "SVD_EXACT", "SVD_RANDOMIZED", "fit_params", "fkk_apply",
    "fkk_basis_from_arrays", "fkk_basis_load", "fkk_noise_scale", "Server", "fkk_basis_math", "fkk_eig_topk", "fkk_refine_basis", "fkk_fit_basis", "fkk_fit_many", "CubeJob", "fkk_gram", "fkk_project",
    "fkk_reconstruct", "fkk_reconstruct_noalloc", "kk_per_spectrum", "conventional_per_spectrum", "fkk_residual", "fkk_philox_normals",
    "launch_count", "lib",
]
