"""Pins of the FP64 resampling reference (the mean fields' map to the
surrogate's 128x64x64 grid) against scipy, the 2x2x2 box mean and closed
forms."""
import numpy as np
import pytest

import oracle.lbm as OL
import oracle.resample as R

scipy_ndimage = pytest.importorskip("scipy.ndimage")


@pytest.mark.parametrize("shape", [(96, 64, 192), (128, 96, 256), (64, 128, 128), (64, 64, 128)])
def test_matches_scipy_linear_zoom_on_the_cell_centred_grid(shape):
    """scipy.ndimage.zoom(order=1, grid_mode=True) maps pixel edges to pixel
    edges, i.e. samples the source at (o + 1/2) n/m - 1/2 (clamped by
    mode='nearest'): the same map, computed by another library."""
    r = np.random.default_rng(3)
    f = r.normal(size=shape)
    out = (64, 64, 128)
    ref = scipy_ndimage.zoom(f, [o / s for o, s in zip(out, shape)], order=1, mode="nearest", grid_mode=True)
    assert ref.shape == out
    assert np.abs(R.resample(f, out) - ref).max() < 1e-12


def test_factor_two_is_the_box_mean_and_factor_one_the_identity():
    r = np.random.default_rng(4)
    f = r.normal(size=(2, 16, 12, 20))
    half = OL.halfres(np.moveaxis(f, 0, -1))                      # 2x2x2 box mean of the oracle
    assert np.abs(R.resample(f, (8, 6, 10)) - np.moveaxis(half, -1, 0)).max() < 1e-14
    assert np.abs(R.resample(f, (16, 12, 20)) - f).max() == 0.0


def test_constants_and_interior_affine_fields_are_reproduced():
    """Linear interpolation reproduces an affine field wherever no sample is
    clamped (downsampling by 3/2 or 2 never clamps), and every row of the
    map sums to 1."""
    for n, m in ((192, 128), (96, 64), (256, 128), (128, 128), (64, 128)):
        A = R.interpolation_matrix(n, m)
        assert np.allclose(A.sum(axis=1), 1.0)
        if m <= n:
            x = np.arange(n, dtype=np.float64)
            o = np.arange(m)
            assert np.abs(A @ x - ((o + 0.5) * n / m - 0.5)).max() < 1e-12
