"""Pins of the FP64 FNO oracle: library FFTs, adjoint identities, exact
special cases and finite differences."""
import math

import numpy as np
import pytest

import oracle.fno as F


def tiny(grid=(8, 6, 10), modes=(3, 2, 3), width=3, layers=2, hidden=5, lift_hidden=4, omega0=30.0):
    return F.FNOConfig(grid=grid, cin=2, width=width, cout=2, modes=modes, layers=layers, hidden=hidden,
                       lift_hidden=lift_hidden, omega0=omega0)


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


# --------------------------------------------------------------------------
# App. B's lift (feed-forward network) and projection (SIREN)
# --------------------------------------------------------------------------
def test_siren_projection_is_periodic_in_its_bias():
    """sin(omega0 (Q1 v + b)) is unchanged when b moves by 2 pi / omega0: the
    frequency factor multiplies the bias as well as Q1 v."""
    cfg = tiny()
    p = F.init_params(cfg, seed=11)
    x = rng(12).normal(size=(2, cfg.cin) + cfg.grid)
    y0 = F.forward(p, x, cfg)
    q = dict(p)
    q["Q1_b"] = p["Q1_b"] + 2 * np.pi / cfg.omega0 * rng(13).integers(-3, 4, size=p["Q1_b"].shape)
    assert np.abs(F.forward(q, x, cfg) - y0).max() < 1e-12 * np.abs(y0).max()
    q["Q1_b"] = p["Q1_b"] + np.pi / cfg.omega0         # half a period flips every hidden unit
    assert np.abs(F.forward(q, x, cfg) - (2 * p["Q2_b"][None, :, None, None, None] - y0)).max() < 1e-12


def test_siren_projection_tends_to_the_linear_map_at_small_frequency():
    """With the output weights scaled by 1/omega0, Q2 sin(omega0 z)/omega0 ->
    Q2 z as omega0 -> 0, with an error that falls as omega0^2 (the cubic term
    of the sine)."""
    base = tiny()
    p = F.init_params(base, seed=14)
    x = rng(15).normal(size=(1, base.cin) + base.grid)
    _, tape = F.forward(p, x, base, keep=True)
    vL = tape["v"][-1]
    lin = F.pointwise(p["Q2_w"], p["Q2_b"], F.pointwise(p["Q1_w"], p["Q1_b"], vL))
    errs = []
    for w0 in (1e-2, 5e-3):
        cfg = tiny(omega0=w0)
        q = dict(p)
        q["Q2_w"] = p["Q2_w"] / w0
        errs.append(np.abs(F.forward(q, x, cfg) - lin).max())
    assert errs[0] < 1e-3 * np.abs(lin).max()
    assert 3.9 < errs[0] / errs[1] < 4.1


def test_lift_is_two_layers_with_gelu_between():
    """Where every hidden pre-activation is large and positive, GELU is the
    identity to rounding (x Phi(x), Phi(9) = 1 - 1e-19), so the lift collapses
    to the affine map P2 (P1 x + b1) + b2; where they are large and negative
    GELU is 0 and the lift is the constant b2."""
    cfg = tiny(layers=1)
    p = F.init_params(cfg, seed=16)
    x = np.abs(rng(17).normal(size=(1, cfg.cin) + cfg.grid))
    for sign in (1.0, -1.0):
        q = dict(p)
        q["P1_w"] = sign * np.abs(p["P1_w"])
        q["P1_b"] = np.full_like(p["P1_b"], sign * 9.0)
        _, tape = F.forward(q, x, cfg, keep=True)
        v0 = tape["v"][0]
        if sign > 0:
            ref = F.pointwise(q["P2_w"], q["P2_b"], F.pointwise(q["P1_w"], q["P1_b"], x))
        else:
            ref = np.broadcast_to(q["P2_b"][None, :, None, None, None], v0.shape)
        assert np.abs(v0 - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())


def test_siren_initialisation_ranges():
    """Sitzmann et al.'s initialisation of the projection: first-layer weights
    within 1/fan_in, output weights within sqrt(6/fan_in)/omega0."""
    cfg = F.FNOConfig(grid=(4, 4, 4), width=32, hidden=128)
    p = F.init_params(cfg, seed=18)
    assert np.abs(p["Q1_w"]).max() <= 1 / 32 and np.abs(p["Q1_w"]).max() > 0.9 / 32
    lim = math.sqrt(6 / 128) / 30
    assert np.abs(p["Q2_w"]).max() <= lim and np.abs(p["Q2_w"]).max() > 0.9 * lim
