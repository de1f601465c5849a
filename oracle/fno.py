"""Plain FP64 reference of the Fourier Neural Operator surrogate (test
infrastructure only; the product path never imports it).

The paper (Sec. 4 and App. B) trains an FNO (Li et al. 2021) that maps the
obstacle mask and Re to the mean flow field.  App. B fixes three parts of it:
the lifting layer is a simple feed-forward network that expands the inputs to
the 32-channel co-domain, the Fourier layers keep a box of low modes, and the
projection is a SIREN (Sitzmann et al. 2020: layers with sine activations
sin(omega0 (W x + b)), omega0 = 30, and their initialisation).  This module
restates that network for fields laid out [batch, channel, z, y, x]:

  lift      a = GELU(P1 x + bP1);  v0 = P2 a + bP2         (cin -> lift_hidden -> width)
  layer l   v_{l+1} = act( K_l v_l + W_l v_l + b_l )       (act = GELU except the last)
            K_l v = IDFT_r( R_l . DFT_r(v) )               (retained modes only)
  project   h = sin(omega0 (Q1 v_L + bQ1));  y = Q2 h + bQ2 (width -> hidden -> cout)

DFT_r is the discrete Fourier transform restricted to the retained modes
kx in [0, mx) U [-mx, 0), ky in [0, my) U [-my, 0), kz in [0, mz) (z is the
real-to-half-complex axis):  V(k) = sum_x v(x) exp(-i theta_k . x),
theta_k . x = 2 pi (kx x / nx + ky y / ny + kz z / nz).
IDFT_r is the inverse of a real field from those modes:
  y(x) = (1/N) Re[ sum_k c_kz G(k) exp(+i theta_k . x) ],  c_0 = c_{nz/2} = 1, else 2.
R_l holds one complex width x width matrix per retained mode:
  G(b, o, k) = sum_i V(b, i, k) R_l(i, o, k).
GELU is the exact form x Phi(x).  The loss is the masked mean square error
sum_{b,c,x} M(b,x) (y - t)^2 / (C * sum M).

Gradients are written by hand; complex gradients use g = dL/dRe + i dL/dIm,
for which a product z = a w gives g_a = g_z conj(w), g_w = g_z conj(a).  The
sine layer's derivative is d sin(omega0 z)/dz = omega0 cos(omega0 z).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

try:
    from scipy.special import erf as _erf
except Exception:                                     # pragma: no cover
    _erf = np.vectorize(math.erf)


@dataclass
class FNOConfig:
    grid: tuple = (64, 64, 128)        # (nz, ny, nx)
    cin: int = 4
    width: int = 32
    cout: int = 4
    modes: tuple = (8, 8, 16)          # (mz, my, mx)
    layers: int = 4
    hidden: int = 128                  # SIREN projection width
    lift_hidden: int = 32              # hidden width of the feed-forward lift
    omega0: float = 30.0               # SIREN frequency factor

    @property
    def nmodes(self):
        mz, my, mx = self.modes
        return mz * 2 * my * 2 * mx


def mode_numbers(cfg):
    """Retained wave numbers along z, y, x."""
    mz, my, mx = cfg.modes
    kz = np.arange(mz)
    ky = np.concatenate([np.arange(my), np.arange(-my, 0)])
    kx = np.concatenate([np.arange(mx), np.arange(-mx, 0)])
    return kz, ky, kx


def _exp_mats(cfg, sign):
    nz, ny, nx = cfg.grid
    kz, ky, kx = mode_numbers(cfg)
    Ez = np.exp(sign * 2j * np.pi * np.outer(kz, np.arange(nz)) / nz)
    Ey = np.exp(sign * 2j * np.pi * np.outer(ky, np.arange(ny)) / ny)
    Ex = np.exp(sign * 2j * np.pi * np.outer(kx, np.arange(nx)) / nx)
    return Ez, Ey, Ex


def c_weights(cfg):
    nz = cfg.grid[0]
    kz = mode_numbers(cfg)[0]
    c = np.full(len(kz), 2.0)
    c[kz == 0] = 1.0
    if nz % 2 == 0:
        c[kz == nz // 2] = 1.0
    return c


def dft_r(v, cfg):
    """Truncated forward DFT: [..., z, y, x] real -> [..., Kz, Ky, Kx] complex."""
    Ez, Ey, Ex = _exp_mats(cfg, -1.0)
    return np.einsum('...zyx,az,by,cx->...abc', v, Ez, Ey, Ex, optimize=True)


def idft_r(G, cfg):
    """Inverse from the retained modes to a real field."""
    Ez, Ey, Ex = _exp_mats(cfg, +1.0)
    N = np.prod(cfg.grid)
    Gc = G * c_weights(cfg)[:, None, None]
    return np.real(np.einsum('...abc,az,by,cx->...zyx', Gc, Ez, Ey, Ex, optimize=True)) / N


def dft_r_adjoint(g, cfg):
    """Adjoint of dft_r: real field from complex mode gradients,
    Re[sum_k g(k) exp(+i theta_k . x)] (no 1/N, no c weights)."""
    Ez, Ey, Ex = _exp_mats(cfg, +1.0)
    return np.real(np.einsum('...abc,az,by,cx->...zyx', g, Ez, Ey, Ex, optimize=True))


def idft_r_adjoint(g, cfg):
    """Adjoint of idft_r: complex mode gradients (c_kz / N) dft_r(g)."""
    N = np.prod(cfg.grid)
    return dft_r(g, cfg) * (c_weights(cfg)[:, None, None] / N)


def gelu(x):
    return 0.5 * x * (1.0 + _erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + _erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def pointwise(w, b, v):
    """[cout, cin] x [B, cin, ...] + b -> [B, cout, ...]."""
    out = np.einsum('oi,bi...->bo...', w, v)
    return out + b.reshape((1, -1) + (1,) * (v.ndim - 2))


def channel_outer(a, b):
    """sum over batch and cells of a[b, o, ...] b[b, i, ...] -> [o, i]."""
    return np.einsum('bon,bin->oi', a.reshape(a.shape[0], a.shape[1], -1), b.reshape(b.shape[0], b.shape[1], -1))


def siren(w, b, v, omega0):
    """SIREN layer: sin(omega0 (W v + b)) and its pre-activation W v + b."""
    z = pointwise(w, b, v)
    return np.sin(omega0 * z), z


def init_params(cfg, seed=0):
    """Deterministic FP64 parameters.  Lift, Fourier-layer pointwise weights
    and biases: uniform(-s, s) with s = 1/sqrt(fan_in); spectral weights
    uniform with scale 1/(width^2) on real and imaginary parts; SIREN
    projection (Sitzmann et al. 2020): first (sine) layer weights uniform
    within 1/fan_in, the last (linear) layer's within sqrt(6/fan_in)/omega0,
    biases within 1/sqrt(fan_in)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    W = cfg.width
    LH = cfg.lift_hidden
    mz, my, mx = cfg.modes

    def u(shape, s):
        return rng.uniform(-s, s, shape)

    p = {"P1_w": u((LH, cfg.cin), 1 / math.sqrt(cfg.cin)), "P1_b": u((LH,), 1 / math.sqrt(cfg.cin)),
         "P2_w": u((W, LH), 1 / math.sqrt(LH)), "P2_b": u((W,), 1 / math.sqrt(LH))}
    for l in range(cfg.layers):
        scale = 1.0 / (W * W)
        p[f"R{l}"] = (rng.uniform(-scale, scale, (W, W, mz, 2 * my, 2 * mx))
                      + 1j * rng.uniform(-scale, scale, (W, W, mz, 2 * my, 2 * mx)))
        p[f"W{l}_w"] = u((W, W), 1 / math.sqrt(W))
        p[f"W{l}_b"] = u((W,), 1 / math.sqrt(W))
    p["Q1_w"] = u((cfg.hidden, W), 1.0 / W)
    p["Q1_b"] = u((cfg.hidden,), 1 / math.sqrt(W))
    p["Q2_w"] = u((cfg.cout, cfg.hidden), math.sqrt(6.0 / cfg.hidden) / cfg.omega0)
    p["Q2_b"] = u((cfg.cout,), 1 / math.sqrt(cfg.hidden))
    return p


def forward(p, x, cfg, keep=False):
    apre = pointwise(p["P1_w"], p["P1_b"], x)                  # feed-forward lift
    a = gelu(apre)
    v = pointwise(p["P2_w"], p["P2_b"], a)
    tape = {"x": x, "apre": apre, "a": a, "v": [v], "pre": [], "Vhat": []}
    for l in range(cfg.layers):
        Vh = dft_r(v, cfg)                                        # [B, i, K]
        G = np.einsum('bi...,io...->bo...', Vh, p[f"R{l}"])
        pre = idft_r(G, cfg) + pointwise(p[f"W{l}_w"], p[f"W{l}_b"], v)
        v = gelu(pre) if l < cfg.layers - 1 else pre
        tape["Vhat"].append(Vh)
        tape["pre"].append(pre)
        tape["v"].append(v)
    h, hpre = siren(p["Q1_w"], p["Q1_b"], v, cfg.omega0)         # SIREN projection
    y = pointwise(p["Q2_w"], p["Q2_b"], h)
    tape.update(hpre=hpre, h=h)
    return (y, tape) if keep else y


def masked_mse(y, t, m):
    """m: [B, z, y, x] weights; mean over channels and weighted cells."""
    d = (y - t) * m[:, None]
    return float((d * (y - t)).sum() / (y.shape[1] * m.sum()))


def backward(p, tape, y, t, m, cfg):
    """Gradients of masked_mse(forward(p, x), t, m) with respect to p."""
    B, C = y.shape[:2]
    g = {}
    gy = 2.0 * (y - t) * m[:, None] / (C * m.sum())
    h, hpre = tape["h"], tape["hpre"]
    g["Q2_w"] = channel_outer(gy, h)
    g["Q2_b"] = gy.sum(axis=tuple(i for i in range(gy.ndim) if i != 1))
    gh = np.einsum('oi,bo...->bi...', p["Q2_w"], gy) * (cfg.omega0 * np.cos(cfg.omega0 * hpre))
    v = tape["v"][-1]
    g["Q1_w"] = channel_outer(gh, v)
    g["Q1_b"] = gh.sum(axis=tuple(i for i in range(gh.ndim) if i != 1))
    gv = np.einsum('oi,bo...->bi...', p["Q1_w"], gh)
    for l in reversed(range(cfg.layers)):
        pre = tape["pre"][l]
        gpre = gv * gelu_grad(pre) if l < cfg.layers - 1 else gv
        vin = tape["v"][l]
        g[f"W{l}_w"] = channel_outer(gpre, vin)
        g[f"W{l}_b"] = gpre.sum(axis=tuple(i for i in range(gpre.ndim) if i != 1))
        gv_point = np.einsum('oi,bo...->bi...', p[f"W{l}_w"], gpre)
        gG = idft_r_adjoint(gpre, cfg)                            # [B, o, K]
        Vh = tape["Vhat"][l]
        g[f"R{l}"] = np.einsum('boklm,biklm->ioklm', gG, np.conj(Vh))
        gVh = np.einsum('bo...,io...->bi...', gG, np.conj(p[f"R{l}"]))
        gv = gv_point + dft_r_adjoint(gVh, cfg)
    a, apre, x = tape["a"], tape["apre"], tape["x"]
    g["P2_w"] = channel_outer(gv, a)
    g["P2_b"] = gv.sum(axis=tuple(i for i in range(gv.ndim) if i != 1))
    ga = np.einsum('oi,bo...->bi...', p["P2_w"], gv) * gelu_grad(apre)
    g["P1_w"] = channel_outer(ga, x)
    g["P1_b"] = ga.sum(axis=tuple(i for i in range(ga.ndim) if i != 1))
    return g


def loss_and_grad(p, x, t, m, cfg):
    y, tape = forward(p, x, cfg, keep=True)
    return masked_mse(y, t, m), backward(p, tape, y, t, m, cfg)


def region_mask(grid, lo=(0.25, 0.25, 0.1), hi=(0.75, 0.75, 0.9)):
    """Inner region of the channel used by the loss: the box
    [(0.2, 0.25, 0.25), (1.8, 0.75, 0.75)] of the (2, 1, 1) domain, i.e. x in
    [0.1, 0.9) of the length and y, z in [0.25, 0.75) of the height (returned
    [z, y, x])."""
    nz, ny, nx = grid
    m = np.zeros(grid)
    m[int(lo[0] * nz):int(hi[0] * nz), int(lo[1] * ny):int(hi[1] * ny), int(lo[2] * nx):int(hi[2] * nx)] = 1.0
    return m


def adam_step(p, g, m1, m2, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (bias-corrected), real and imaginary parts separately."""
    for k in p:
        m1[k] = b1 * m1[k] + (1 - b1) * g[k]
        if np.iscomplexobj(g[k]):
            sq = g[k].real ** 2 + 1j * g[k].imag ** 2
        else:
            sq = g[k] ** 2
        m2[k] = b2 * m2[k] + (1 - b2) * sq
        mh = m1[k] / (1 - b1 ** step)
        vh = m2[k] / (1 - b2 ** step)
        if np.iscomplexobj(p[k]):
            p[k] = p[k] - lr * (mh.real / (np.sqrt(vh.real) + eps) + 1j * mh.imag / (np.sqrt(vh.imag) + eps))
        else:
            p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
    return p
