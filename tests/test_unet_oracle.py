"""Pins of the FP64 U-Net reference (oracle/unet.py) against library
routines, closed forms and finite differences."""
import numpy as np
import pytest

import oracle.unet as U

scipy_signal = pytest.importorskip("scipy.signal")
scipy_ndimage = pytest.importorskip("scipy.ndimage")


def test_conv3_is_the_zero_padded_cross_correlation():
    r = np.random.default_rng(0)
    x = r.normal(size=(2, 3, 4, 5, 6))
    w = r.normal(size=(4, 3, 3, 3, 3))
    y = U.conv3(x, w)
    ref = np.zeros_like(y)
    for b in range(2):
        for o in range(4):
            for i in range(3):
                ref[b, o] += scipy_signal.correlate(x[b, i], w[o, i], mode="same", method="direct")
    assert np.abs(y - ref).max() < 1e-12


def test_upsampling_is_scipy_linear_zoom_with_cell_centred_grid():
    r = np.random.default_rng(1)
    x = r.normal(size=(1, 2, 3, 4, 5))
    y = U.up2(x)
    for c in range(2):
        ref = scipy_ndimage.zoom(x[0, c], 2, order=1, mode="nearest", grid_mode=True)
        assert np.abs(y[0, c] - ref).max() < 1e-12


def test_upsampling_closed_forms():
    # [a, b] -> [a, 3a/4 + b/4, a/4 + 3b/4, b]; a constant stays constant;
    # a field linear in x is reproduced away from the clamped end samples
    m = U.upsample_matrix(2)
    assert np.allclose(m @ np.array([1.0, 0.0]), [1.0, 0.75, 0.25, 0.0])
    assert np.allclose(U.upsample_matrix(7).sum(axis=1), 1.0)
    x = np.arange(6.0)
    y = U.upsample_matrix(6) @ x
    o = np.arange(1, 11)
    assert np.allclose(y[o], (o + 0.5) / 2 - 0.5)


def test_maxpool_is_the_window_maximum():
    r = np.random.default_rng(2)
    x = r.normal(size=(2, 3, 4, 6, 8))
    y, arg = U.maxpool2(x)
    ref = x.reshape(2, 3, 2, 2, 3, 2, 4, 2).max(axis=(3, 5, 7))
    assert np.array_equal(y, ref)
    # the gradient lands on the maximum of each window only
    g = U.maxpool2_backward(arg, np.ones_like(y), x.shape)
    assert g.sum() == y.size and np.array_equal(x[g == 1].reshape(-1).size, y.size)
    assert np.all(x[g == 1] >= np.repeat(np.repeat(np.repeat(y, 2, 2), 2, 3), 2, 4)[g == 1])


def test_batchnorm_normalises_each_channel():
    r = np.random.default_rng(3)
    x = 3.0 + 2.0 * r.normal(size=(3, 4, 2, 3, 5))
    y, _ = U.batchnorm(x, np.ones(4), np.zeros(4))
    assert np.abs(y.mean(axis=(0, 2, 3, 4))).max() < 1e-12
    assert np.abs(y.var(axis=(0, 2, 3, 4)) - 1.0).max() < 1e-5     # eps = 1e-5 in the denominator
    g, b = np.array([1.0, 2.0, 0.5, -1.0]), np.array([0.0, 1.0, -2.0, 3.0])
    y2, _ = U.batchnorm(x, g, b)
    assert np.allclose(y2, g[None, :, None, None, None] * y + b[None, :, None, None, None])


def _tiny():
    cfg = U.UNetConfig(grid=(16, 16, 32), cin=2, cout=2, channels=(2, 3, 3, 4), bottleneck=4)
    r = np.random.default_rng(4)
    x = r.normal(size=(2, cfg.cin) + cfg.grid)
    t = r.uniform(size=(2, cfg.cout) + cfg.grid)
    m = (r.uniform(size=(2,) + cfg.grid) < 0.7).astype(float)
    p = U.init_params(cfg, seed=5)
    # non-trivial normalisation parameters, so that their gradients are tested too
    for k in p:
        if k.endswith("_g"):
            p[k] = 1.0 + 0.3 * r.normal(size=p[k].shape)
        if k.endswith("_b"):
            p[k] = 0.2 * r.normal(size=p[k].shape)
    return cfg, x, t, m, p


def test_forward_shapes_and_range():
    cfg, x, t, m, p = _tiny()
    y = U.forward(p, x, cfg)
    assert y.shape == (2, cfg.cout) + cfg.grid
    assert np.all((y > 0) & (y < 1))


def test_backward_matches_central_differences():
    cfg, x, t, m, p = _tiny()
    L, g = U.loss_and_grad(p, x, t, m, cfg)
    r = np.random.default_rng(6)
    # a small step: a shift of a whole channel moves thousands of values, and
    # a step of 1e-6 already carries some of them across a ReLU kink or a
    # max-pooling switch (the difference quotient then drifts by ~0.2 %)
    h = 1e-7
    for k in sorted(p):
        flat = p[k].reshape(-1)
        for j in r.choice(flat.size, size=min(2, flat.size), replace=False):
            old = flat[j]
            flat[j] = old + h
            Lp = U.masked_mse(U.forward(p, x, cfg), t, m)
            flat[j] = old - h
            Lm = U.masked_mse(U.forward(p, x, cfg), t, m)
            flat[j] = old
            fd = (Lp - Lm) / (2 * h)
            an = g[k].reshape(-1)[j]
            assert abs(fd - an) <= 1e-4 * abs(fd) + 1e-9, (k, j, fd, an)
    # and the input gradient
    xf = x.reshape(-1)
    for j in r.choice(xf.size, size=4, replace=False):
        old = xf[j]
        xf[j] = old + h
        Lp = U.masked_mse(U.forward(p, x, cfg), t, m)
        xf[j] = old - h
        Lm = U.masked_mse(U.forward(p, x, cfg), t, m)
        xf[j] = old
        assert abs((Lp - Lm) / (2 * h) - g["input"].reshape(-1)[j]) <= 1e-4 * abs(g["input"].reshape(-1)[j]) + 1e-9


def test_work_of_the_paper_configuration():
    # 128x64x64 grid, 4 -> [32, 64, 128, 256] -> 512 -> ... -> 4: about 150
    # GMAC per sample forward, counted from the layer list
    macs = U.macs(U.UNetConfig())
    assert 1.4e11 < macs < 1.7e11
