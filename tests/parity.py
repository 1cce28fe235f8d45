"""Comparison measure of the parity tests (CUDA path against the oracle).

rel(a, b) is element-wise: the largest point error relative to the largest reference
magnitude, max_i |a_i - b_i| / max_i |b_i|. A few wrong points (a halo or a cluster-chunk
seam) therefore show at their own size instead of being averaged over the vector. The
norm-wise relative error ||a - b||_2 / ||b||_2 is taken as well and the larger of the two
is returned, so a tolerance on rel() bounds both.
"""
import numpy as np


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    assert a.shape == b.shape, (a.shape, b.shape)
    if a.size == 0:
        return 0.0
    if not (np.all(np.isfinite(a)) and np.all(np.isfinite(b))):
        return float("inf")
    pointwise = np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)
    normwise = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)
    return float(max(pointwise, normwise))
