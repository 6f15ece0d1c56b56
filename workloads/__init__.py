"""Seeded synthetic inputs for the GenCD hot path.

This package holds no arithmetic of the method itself: it only draws sparse
design matrices, planted weights and labels shaped like the paper's text-like
data sets (Section 4.4).  The FP64 oracle and the CUDA library both consume the
arrays it returns; neither imports the other.
"""

from .synthetic import (  # noqa: F401
    Problem,
    uniform_problem,
    zipf_problem,
    config1,
    config2,
    config2_scaled,
    config3,
    binarized,
    config4,
    cv_folds,
    lambda_grid,
    row_subset,
    serving_stream,
    tiny_problem,
    csc_from_dense,
)
