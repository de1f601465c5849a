"""Plain FP64 reference of the resampling of mean fields to the surrogate's
grid (test infrastructure only; the product path never imports it).

App. B: the simulated fields (on each geometry's own grid) are scaled down to
128x64x64 before training.  Reading: trilinear interpolation on cell centres.
Output cell o of an axis with n source and m target cells samples the source
at s = (o + 1/2) n / m - 1/2, clamped to [0, n - 1], between the cells
floor(s) and floor(s) + 1 with weights 1 - (s - floor(s)) and s - floor(s).
A factor of 2 is the 2-cell mean, a factor of 1 the identity.  The 3D map is
the product of the three 1D maps (separable).
"""
from __future__ import annotations

import numpy as np


def interpolation_matrix(n: int, m: int) -> np.ndarray:
    """[m, n] matrix of the 1D cell-centred linear resampling n -> m."""
    A = np.zeros((m, n))
    for o in range(m):
        s = (o + 0.5) * n / m - 0.5
        s = min(max(s, 0.0), n - 1.0)
        i0 = int(np.floor(s))
        t = s - i0
        i1 = min(i0 + 1, n - 1)
        A[o, i0] += 1.0 - t
        A[o, i1] += t
    return A


def resample(field, out_shape):
    """field [..., nz, ny, nx] -> [..., mz, my, mx] (out_shape = (mz, my, mx))."""
    f = np.asarray(field, dtype=np.float64)
    nz, ny, nx = f.shape[-3:]
    mz, my, mx = out_shape
    Az, Ay, Ax = interpolation_matrix(nz, mz), interpolation_matrix(ny, my), interpolation_matrix(nx, mx)
    return np.einsum('az,by,cx,...zyx->...abc', Az, Ay, Ax, f, optimize=True)
