"""Pins of the FP64 FNO oracle: library FFTs, adjoint identities, exact
special cases and finite differences."""
import math

import numpy as np
import pytest

import oracle.fno as F


def tiny(grid=(8, 6, 10), modes=(3, 2, 3), width=3, layers=2, hidden=5):
    return F.FNOConfig(grid=grid, cin=2, width=width, cout=2, modes=modes, layers=layers, hidden=hidden)


def rng(s=0):
    return np.random.Generator(np.random.PCG64(s))


def test_truncated_dft_matches_numpy_rfftn():
    cfg = tiny()
    v = rng(1).normal(size=(2, 3) + cfg.grid)
    V = F.dft_r(v, cfg)
    full = np.fft.rfftn(v, axes=(-1, -2, -3))            # rfft along z (the last listed axis)
    kz, ky, kx = F.mode_numbers(cfg)
    ref = full[..., kz[:, None, None], ky[None, :, None], kx[None, None, :]]
    assert np.abs(V - ref).max() < 1e-11


def test_inverse_matches_numpy_irfftn_of_truncated_spectrum():
    cfg = tiny()
    nz, ny, nx = cfg.grid
    G = rng(2).normal(size=(2, 3, cfg.modes[0], 2 * cfg.modes[1], 2 * cfg.modes[2])) \
        + 1j * rng(3).normal(size=(2, 3, cfg.modes[0], 2 * cfg.modes[1], 2 * cfg.modes[2]))
    full = np.zeros((2, 3, nz // 2 + 1, ny, nx), complex)
    kz, ky, kx = F.mode_numbers(cfg)
    full[..., kz[:, None, None], ky[None, :, None], kx[None, None, :]] = G
    ref = np.fft.irfftn(full, s=(nx, ny, nz), axes=(-1, -2, -3))
    assert np.abs(F.idft_r(G, cfg) - ref).max() < 1e-12


def test_full_spectrum_round_trip_and_identity_layer():
    """All modes kept (Nyquist weight 1): IDFT_r(DFT_r(v)) = v, so a spectral
    layer whose matrices are the identity is the identity map."""
    grid = (6, 4, 8)
    cfg = F.FNOConfig(grid=grid, cin=1, width=3, cout=1, modes=(grid[0] // 2 + 1, grid[1] // 2, grid[2] // 2),
                      layers=1, hidden=2)
    v = rng(4).normal(size=(2, 3) + grid)
    assert np.abs(F.idft_r(F.dft_r(v, cfg), cfg) - v).max() < 1e-12
    R = np.zeros((3, 3) + F.dft_r(v, cfg).shape[2:], complex)
    for i in range(3):
        R[i, i] = 1.0
    G = np.einsum('bi...,io...->bo...', F.dft_r(v, cfg), R)
    assert np.abs(F.idft_r(G, cfg) - v).max() < 1e-12


def test_parseval_on_the_half_spectrum():
    grid = (6, 4, 8)
    cfg = F.FNOConfig(grid=grid, modes=(4, 2, 4))
    v = rng(5).normal(size=grid)
    V = F.dft_r(v, cfg)
    c = F.c_weights(cfg)[:, None, None]
    assert abs((v ** 2).sum() - (c * np.abs(V) ** 2).sum() / v.size) < 1e-10


def test_adjoints_by_dot_products():
    cfg = tiny()
    r = rng(6)
    v = r.normal(size=(2, 3) + cfg.grid)
    shape = (2, 3, cfg.modes[0], 2 * cfg.modes[1], 2 * cfg.modes[2])
    g = r.normal(size=shape) + 1j * r.normal(size=shape)
    lhs = np.real(np.sum(np.conj(g) * F.dft_r(v, cfg)))
    rhs = np.sum(v * F.dft_r_adjoint(g, cfg))
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)
    G = r.normal(size=shape) + 1j * r.normal(size=shape)
    w = r.normal(size=(2, 3) + cfg.grid)
    lhs2 = np.sum(w * F.idft_r(G, cfg))
    rhs2 = np.real(np.sum(np.conj(F.idft_r_adjoint(w, cfg)) * G))
    assert abs(lhs2 - rhs2) < 1e-10 * abs(lhs2)


def test_gelu_values_and_derivative():
    x = np.linspace(-4, 4, 81)
    ref = np.array([0.5 * t * (1 + math.erf(t / math.sqrt(2))) for t in x])
    assert np.abs(F.gelu(x) - ref).max() < 1e-15
    h = 1e-6
    fd = (F.gelu(x + h) - F.gelu(x - h)) / (2 * h)
    assert np.abs(F.gelu_grad(x) - fd).max() < 1e-8


def test_gradients_match_central_differences():
    cfg = tiny()
    p = F.init_params(cfg, seed=7)
    for k in p:                                  # larger spectral weights exercise the path
        if k.startswith("R"):
            p[k] = p[k] * 30
    r = rng(8)
    B = 2
    x = r.normal(size=(B, cfg.cin) + cfg.grid)
    t = r.normal(size=(B, cfg.cout) + cfg.grid)
    m = (r.uniform(size=(B,) + cfg.grid) < 0.7).astype(float)
    L0, g = F.loss_and_grad(p, x, t, m, cfg)
    h = 1e-6
    for k, arr in p.items():
        flat = arr.reshape(-1)
        idx = r.choice(flat.size, min(6, flat.size), replace=False)
        parts = [(1.0, "re")] + ([(1j, "im")] if np.iscomplexobj(arr) else [])
        for i in idx:
            for unit, part in parts:
                q = {kk: vv.copy() for kk, vv in p.items()}
                q[k].reshape(-1)[i] += h * unit
                Lp = F.masked_mse(F.forward(q, x, cfg), t, m)
                q[k].reshape(-1)[i] -= 2 * h * unit
                Lm = F.masked_mse(F.forward(q, x, cfg), t, m)
                fd = (Lp - Lm) / (2 * h)
                an = g[k].reshape(-1)[i]
                an = an.real if part == "re" else an.imag
                assert abs(an - fd) <= 1e-6 * max(1e-3, abs(fd)), (k, i, part, an, fd)


def test_first_adam_step_is_lr_times_sign():
    p = {"a": np.array([1.0, -2.0, 3.0]), "c": np.array([1 + 1j])}
    g = {"a": np.array([0.5, -1e-3, 2.0]), "c": np.array([-0.3 + 0.7j])}
    m1 = {k: np.zeros_like(v) for k, v in p.items()}
    m2 = {k: np.zeros_like(v) for k, v in p.items()}
    q = F.adam_step({k: v.copy() for k, v in p.items()}, g, m1, m2, 1, 0.01)
    assert np.allclose(q["a"], p["a"] - 0.01 * np.sign(g["a"]), atol=1e-9)
    assert np.allclose(q["c"], p["c"] - 0.01 * (np.sign(g["c"].real) + 1j * np.sign(g["c"].imag)), atol=1e-9)


def test_region_mask_box():
    m = F.region_mask((64, 64, 128))
    z, y, x = np.nonzero(m)
    assert (x.min(), x.max() + 1) == (12, 115) and (y.min(), y.max() + 1) == (16, 48)
    assert (z.min(), z.max() + 1) == (16, 48)
