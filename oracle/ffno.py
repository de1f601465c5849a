"""Plain FP64 reference of the factorised Fourier Neural Operator (FFNO)
surrogate (test infrastructure only; the product path never imports it).

The paper's Table 2 compares an FFNO (Tran et al., "Factorized Fourier
Neural Operators") with the FNO, a hybrid and the U-Net; its appendix on the
baselines says the FFNO follows Tran et al.'s structure, with the FNO models'
32 x 16 x 16 modes, 32 channels, feed-forward lift and SIREN projection.  The
FFNO replaces the FNO's 3-D spectral convolution by a sum of 1-D spectral
convolutions, one per axis, and puts a feed-forward block with a residual
connection after it.  For fields laid out [batch, channel, z, y, x]:

  lift      a = GELU(P1 x + bP1);  v0 = P2 a + bP2             (as the FNO)
  layer l   u = sum_{d in z, y, x} IDFT_d( R_{l,d} . DFT_d(v_l) )
            v_{l+1} = v_l + F2_l GELU(F1_l u + b1_l) + b2_l
  project   h = sin(omega0 (Q1 v_L + bQ1));  y = Q2 h + bQ2     (as the FNO)

DFT_d is the real-input discrete Fourier transform along axis d alone,
restricted to the first m_d wave numbers k in [0, m_d):
  V(k) = sum_n v(n) exp(-2 pi i k n / N_d);
IDFT_d the inverse to a real field from those modes,
  u(n) = (1/N_d) Re[ sum_k c_k W(k) exp(+2 pi i k n / N_d) ],
  c_0 = 1, c_{N_d/2} = 1 (N_d even), otherwise c_k = 2;
R_{l,d} holds one complex width x width matrix per wave number of axis d:
  W(b, o, ..., k) = sum_i V(b, i, ..., k) R_{l,d}(i, o, k).

Readings where the paper and the cited structure leave a choice (listed in
the design notes): GELU in the feed-forward block (the FNO's activation), its
hidden width a parameter (default the channel width), no activation after
the residual sum, the lift and the projection of the FNO.

Gradients are written by hand with the FNO oracle's complex convention
(g = dL/dRe + i dL/dIm).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import fno as _fno

gelu, gelu_grad = _fno.gelu, _fno.gelu_grad
pointwise, channel_outer, siren = _fno.pointwise, _fno.channel_outer, _fno.siren
masked_mse, adam_step = _fno.masked_mse, _fno.adam_step

AXES = ("z", "y", "x")


@dataclass
class FFNOConfig:
    grid: tuple = (64, 64, 128)        # (nz, ny, nx)
    cin: int = 4
    width: int = 32
    cout: int = 4
    modes: tuple = (16, 16, 32)        # (mz, my, mx): wave numbers kept along each axis
    layers: int = 4
    ff_hidden: int = 32                # hidden width of the feed-forward block
    hidden: int = 128                  # SIREN projection width
    lift_hidden: int = 32              # hidden width of the feed-forward lift
    omega0: float = 30.0               # SIREN frequency factor


def _axis(v, d):
    """Array axis of field axis d (0 = z, 1 = y, 2 = x) for [B, C, z, y, x]."""
    return v.ndim - 3 + d


def c_weights(n, m):
    """Weights c_k of the real inverse for k in [0, m) on n samples."""
    c = np.full(m, 2.0)
    c[0] = 1.0
    if n % 2 == 0 and m > n // 2:
        c[n // 2] = 1.0
    return c


def exp_mat(n, m, sign):
    """[m, n]: exp(sign 2 pi i k j / n)."""
    return np.exp(sign * 2j * np.pi * np.outer(np.arange(m), np.arange(n)) / n)


def dft_axis(v, d, m):
    """Truncated forward DFT of a real field along field axis d: the sample
    axis is replaced by the m wave numbers."""
    a = _axis(v, d)
    E = exp_mat(v.shape[a], m, -1.0)
    return np.moveaxis(np.tensordot(np.moveaxis(v, a, -1), E, axes=([-1], [1])), -1, a)


def idft_axis(G, d, n):
    """Real field on n samples along field axis d from its first wave numbers."""
    a = _axis(G, d)
    m = G.shape[a]
    E = exp_mat(n, m, +1.0) * c_weights(n, m)[:, None]
    return np.real(np.moveaxis(np.tensordot(np.moveaxis(G, a, -1), E, axes=([-1], [0])), -1, a)) / n


def dft_axis_adjoint(g, d, n):
    """Adjoint of dft_axis for a real input: Re[sum_k g(k) exp(+2 pi i k j / n)]."""
    a = _axis(g, d)
    m = g.shape[a]
    E = exp_mat(n, m, +1.0)
    return np.real(np.moveaxis(np.tensordot(np.moveaxis(g, a, -1), E, axes=([-1], [0])), -1, a))


def idft_axis_adjoint(g, d, m):
    """Adjoint of idft_axis: complex mode gradients (c_k / n) dft_axis(g)."""
    a = _axis(g, d)
    n = g.shape[a]
    w = c_weights(n, m) / n
    return dft_axis(g, d, m) * w.reshape((-1,) + (1,) * (g.ndim - 1 - a))


def mix(V, R, d):
    """W(b, o, ..., k) = sum_i V(b, i, ..., k) R(i, o, k), k on field axis d."""
    a = _axis(V, d)
    Vm = np.moveaxis(V, a, -1)                               # [B, i, ..., k]
    W = np.einsum('bi...k,iok->bo...k', Vm, R)
    return np.moveaxis(W, -1, a)


def spectral(v, Rs, cfg):
    """u = sum_d IDFT_d(R_d . DFT_d(v)); also the per-axis spectra."""
    u = np.zeros(v.shape[:1] + (v.shape[1],) + v.shape[2:])
    spectra = []
    for d in range(3):
        V = dft_axis(v, d, cfg.modes[d])
        u = u + idft_axis(mix(V, Rs[d], d), d, cfg.grid[d])
        spectra.append(V)
    return u, spectra


def init_params(cfg, seed=0):
    """Deterministic FP64 parameters: lift and SIREN projection as the FNO
    oracle draws them; per layer and axis the spectral weights uniform with
    scale 1/width^2 on real and imaginary parts; feed-forward weights and
    biases uniform(-s, s), s = 1/sqrt(fan_in)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    W, H, LH = cfg.width, cfg.ff_hidden, cfg.lift_hidden

    def u(shape, s):
        return rng.uniform(-s, s, shape)

    p = {"P1_w": u((LH, cfg.cin), 1 / math.sqrt(cfg.cin)), "P1_b": u((LH,), 1 / math.sqrt(cfg.cin)),
         "P2_w": u((W, LH), 1 / math.sqrt(LH)), "P2_b": u((W,), 1 / math.sqrt(LH))}
    for l in range(cfg.layers):
        scale = 1.0 / (W * W)
        for d, name in enumerate(AXES):
            m = cfg.modes[d]
            p[f"R{l}{name}"] = rng.uniform(-scale, scale, (W, W, m)) + 1j * rng.uniform(-scale, scale, (W, W, m))
        p[f"F{l}a_w"] = u((H, W), 1 / math.sqrt(W))
        p[f"F{l}a_b"] = u((H,), 1 / math.sqrt(W))
        p[f"F{l}b_w"] = u((W, H), 1 / math.sqrt(H))
        p[f"F{l}b_b"] = u((W,), 1 / math.sqrt(H))
    p["Q1_w"] = u((cfg.hidden, W), 1.0 / W)
    p["Q1_b"] = u((cfg.hidden,), 1 / math.sqrt(W))
    p["Q2_w"] = u((cfg.cout, cfg.hidden), math.sqrt(6.0 / cfg.hidden) / cfg.omega0)
    p["Q2_b"] = u((cfg.cout,), 1 / math.sqrt(cfg.hidden))
    return p


def layer_weights(p, l):
    return [p[f"R{l}{name}"] for name in AXES]


def forward(p, x, cfg, keep=False):
    apre = pointwise(p["P1_w"], p["P1_b"], x)                  # feed-forward lift
    a = gelu(apre)
    v = pointwise(p["P2_w"], p["P2_b"], a)
    tape = {"x": x, "apre": apre, "a": a, "v": [v], "u": [], "z": [], "hff": [], "spectra": []}
    for l in range(cfg.layers):
        u, spectra = spectral(v, layer_weights(p, l), cfg)
        z = pointwise(p[f"F{l}a_w"], p[f"F{l}a_b"], u)
        hff = gelu(z)
        v = v + pointwise(p[f"F{l}b_w"], p[f"F{l}b_b"], hff)
        for k, val in (("u", u), ("z", z), ("hff", hff), ("spectra", spectra), ("v", v)):
            tape[k].append(val)
    h, hpre = siren(p["Q1_w"], p["Q1_b"], v, cfg.omega0)         # SIREN projection
    y = pointwise(p["Q2_w"], p["Q2_b"], h)
    tape.update(hpre=hpre, h=h)
    return (y, tape) if keep else y


def _bias_grad(g):
    return g.sum(axis=tuple(i for i in range(g.ndim) if i != 1))


def backward(p, tape, y, t, m, cfg):
    """Gradients of masked_mse(forward(p, x), t, m) with respect to p."""
    C = y.shape[1]
    g = {}
    gy = 2.0 * (y - t) * m[:, None] / (C * m.sum())
    h, hpre = tape["h"], tape["hpre"]
    g["Q2_w"] = channel_outer(gy, h)
    g["Q2_b"] = _bias_grad(gy)
    gh = np.einsum('oi,bo...->bi...', p["Q2_w"], gy) * (cfg.omega0 * np.cos(cfg.omega0 * hpre))
    g["Q1_w"] = channel_outer(gh, tape["v"][-1])
    g["Q1_b"] = _bias_grad(gh)
    gv = np.einsum('oi,bo...->bi...', p["Q1_w"], gh)
    for l in reversed(range(cfg.layers)):
        u, z, hff, spectra = tape["u"][l], tape["z"][l], tape["hff"][l], tape["spectra"][l]
        # v_{l+1} = v_l + F2 GELU(F1 u + b1) + b2
        g[f"F{l}b_w"] = channel_outer(gv, hff)
        g[f"F{l}b_b"] = _bias_grad(gv)
        gz = np.einsum('oi,bo...->bi...', p[f"F{l}b_w"], gv) * gelu_grad(z)
        g[f"F{l}a_w"] = channel_outer(gz, u)
        g[f"F{l}a_b"] = _bias_grad(gz)
        gu = np.einsum('oi,bo...->bi...', p[f"F{l}a_w"], gz)
        gin = gv.copy()                                            # the residual path
        for d, name in enumerate(AXES):
            R = p[f"R{l}{name}"]
            a = _axis(gu, d)
            gW = idft_axis_adjoint(gu, d, cfg.modes[d])            # [B, o, ..., k]
            Wm, Vm = np.moveaxis(gW, a, -1), np.moveaxis(spectra[d], a, -1)
            Wf = Wm.reshape(Wm.shape[0], Wm.shape[1], -1, Wm.shape[-1])   # [B, o, positions, k]
            Vf = Vm.reshape(Vm.shape[0], Vm.shape[1], -1, Vm.shape[-1])
            g[f"R{l}{name}"] = np.einsum('bopk,bipk->iok', Wf, np.conj(Vf))
            gV = np.moveaxis(np.einsum('bo...k,iok->bi...k', Wm, np.conj(R)), -1, a)
            gin = gin + dft_axis_adjoint(gV, d, cfg.grid[d])
        gv = gin
    a, apre, x = tape["a"], tape["apre"], tape["x"]
    g["P2_w"] = channel_outer(gv, a)
    g["P2_b"] = _bias_grad(gv)
    ga = np.einsum('oi,bo...->bi...', p["P2_w"], gv) * gelu_grad(apre)
    g["P1_w"] = channel_outer(ga, x)
    g["P1_b"] = _bias_grad(ga)
    g["input"] = np.einsum('oi,bo...->bi...', p["P1_w"], ga)
    return g


def loss_and_grad(p, x, t, m, cfg):
    y, tape = forward(p, x, cfg, keep=True)
    return masked_mse(y, t, m), backward(p, tape, y, t, m, cfg)
