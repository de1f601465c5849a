"""Pins of the FP64 FFNO reference (oracle/ffno.py) against what the
mathematics fixes: the per-axis transforms against numpy's real FFT, exact
reconstruction from the full half spectrum, the adjoint identities, closed
forms of the factorised spectral operator, the residual block's identity
case, and the hand backward against central differences."""
import numpy as np
import pytest

from oracle import ffno as F


def tiny(layers=2):
    return F.FFNOConfig(grid=(6, 5, 8), cin=2, width=3, cout=2, modes=(2, 3, 4), layers=layers, ff_hidden=4,
                        hidden=5, lift_hidden=3)


def field(shape, seed):
    return np.random.default_rng(seed).normal(size=shape)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_axis_transform_is_the_truncated_real_fft(d):
    v = field((2, 3, 6, 5, 8), 1)
    m = 3
    ref = np.take(np.fft.rfft(v, axis=2 + d), np.arange(m), axis=2 + d)
    assert np.allclose(F.dft_axis(v, d, m), ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_full_half_spectrum_reconstructs_the_field(d):
    v = field((1, 2, 6, 5, 8), 2)                      # even (6, 8) and odd (5) lengths
    n = v.shape[2 + d]
    assert np.allclose(F.idft_axis(F.dft_axis(v, d, n // 2 + 1), d, n), v, rtol=0, atol=1e-12)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_adjoint_identities(d):
    v = field((2, 3, 6, 5, 8), 3)
    n, m = v.shape[2 + d], 3
    shape = list(v.shape)
    shape[2 + d] = m
    g = field(shape, 4) + 1j * field(shape, 5)
    # <DFT v, g> = <v, DFT^T g> (real inner product of complex numbers)
    lhs = np.real(np.sum(np.conj(F.dft_axis(v, d, m)) * g))
    rhs = np.sum(v * F.dft_axis_adjoint(g, d, n))
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)
    # <IDFT G, u> = <G, IDFT^T u>
    u = field(v.shape, 6)
    lhs = np.sum(F.idft_axis(g, d, n) * u)
    rhs = np.real(np.sum(np.conj(g) * F.idft_axis_adjoint(u, d, m)))
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


def test_identity_weights_on_every_mode_give_three_times_the_field():
    cfg = F.FFNOConfig(grid=(6, 5, 8), width=3, modes=(4, 3, 5))      # every wave number of each axis
    v = field((2, 3) + cfg.grid, 7)
    eye = [np.repeat(np.eye(3)[:, :, None], m, axis=2).astype(complex) for m in cfg.modes]
    u, _ = F.spectral(v, eye, cfg)
    assert np.allclose(u, 3.0 * v, rtol=0, atol=1e-12)


def test_branch_of_an_axis_the_field_is_constant_along():
    """A field constant along y: DFT_y keeps only k = 0 (ny times the field),
    so the y branch alone is the real part of R_y(k = 0) mixing the channels."""
    cfg = tiny()
    v = np.repeat(field((2, 3, 6, 1, 8), 8), 5, axis=3)
    r = np.random.default_rng(9)
    Ry = r.normal(size=(3, 3, 3)) + 1j * r.normal(size=(3, 3, 3))
    zero = [np.zeros((3, 3, m), complex) for m in cfg.modes]
    u, _ = F.spectral(v, [zero[0], Ry, zero[2]], cfg)
    ref = np.einsum('bizyx,io->bozyx', v, Ry[:, :, 0].real)
    assert np.allclose(u, ref, rtol=0, atol=1e-12)


def test_zero_feed_forward_output_makes_every_layer_the_identity():
    cfg = tiny()
    p = F.init_params(cfg, seed=1)
    for l in range(cfg.layers):
        p[f"F{l}b_w"][:] = 0.0
        p[f"F{l}b_b"][:] = 0.0
    x = field((2, cfg.cin) + cfg.grid, 10)
    v0 = F.pointwise(p["P2_w"], p["P2_b"], F.gelu(F.pointwise(p["P1_w"], p["P1_b"], x)))
    h, _ = F.siren(p["Q1_w"], p["Q1_b"], v0, cfg.omega0)
    assert np.allclose(F.forward(p, x, cfg), F.pointwise(p["Q2_w"], p["Q2_b"], h), rtol=0, atol=1e-13)


def test_gradients_match_central_differences():
    """Directional derivatives along a random direction of every parameter
    group and of the input."""
    cfg = tiny()
    p = F.init_params(cfg, seed=2)
    r = np.random.default_rng(11)
    x = r.normal(size=(2, cfg.cin) + cfg.grid)
    t = r.normal(size=(2, cfg.cout) + cfg.grid)
    m = (r.uniform(size=(2,) + cfg.grid) < 0.7).astype(float)
    _, g = F.loss_and_grad(p, x, t, m, cfg)
    h = 1e-5
    for k in list(p) + ["input"]:
        base = x if k == "input" else p[k]
        dirn = r.normal(size=base.shape)
        if np.iscomplexobj(base):
            dirn = dirn + 1j * r.normal(size=base.shape)

        def loss(s):
            q = dict(p)
            if k == "input":
                return F.masked_mse(F.forward(p, x + s * dirn, cfg), t, m)
            q[k] = p[k] + s * dirn
            return F.masked_mse(F.forward(q, x, cfg), t, m)

        fd = (loss(h) - loss(-h)) / (2 * h)
        an = float(np.real(np.sum(np.conj(g[k]) * dirn)))
        assert abs(fd - an) <= 1e-6 * max(abs(fd), 1e-8), (k, fd, an)
