"""Plain FP64 reference of the U-Net surrogate (test infrastructure only;
the product path never imports it).

The paper's appendix on the baseline models describes its U-Net, the best
of its surrogates (Sec. 4, Table 2): a 3-D encoder-decoder with skip
connections.  The encoder has four stages of 32, 64, 128 and 256 channels,
each two convolution blocks (convolution, batch normalisation, ReLU)
followed by max-pooling; the bottleneck has 512 channels; the decoder
mirrors the encoder, up-sampling by trilinear interpolation and
concatenating the skip connection; a 1x1x1 convolution with a sigmoid gives
the output channels.  Fields are laid out [batch, channel, z, y, x].

Readings, where the paper is silent:
  * convolutions 3x3x3, zero padding 1, stride 1, no bias (the batch
    normalisation that follows supplies the shift);
  * batch normalisation with the statistics of the batch over
    (batch, z, y, x) (training mode), biased variance, eps = 1e-5, per-channel
    scale gamma and shift beta;
  * max-pooling 2x2x2 with stride 2 (grid sides divisible by 16);
  * trilinear up-sampling by 2 with cell-centred samples: output sample o
    along an axis of n input samples sits at s = (o + 1/2)/2 - 1/2 in input
    coordinates, clamped to [0, n - 1], and interpolates linearly between
    floor(s) and floor(s) + 1;
  * decoder stage d: the up-sampled output of the stage below, concatenated
    after the encoder's skip output of stage d (channels: skip first), then
    two blocks to the stage's channel count;
  * output: 1x1x1 convolution with bias, then the sigmoid; the loss is the
    masked mean square error of the FNO reference (oracle.fno.masked_mse).

Gradients are written by hand (reverse order of the forward tape).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import fno as _fno

EPS = 1e-5


@dataclass
class UNetConfig:
    grid: tuple = (64, 64, 128)            # (nz, ny, nx)
    cin: int = 4
    cout: int = 4
    channels: tuple = (32, 64, 128, 256)   # encoder stages
    bottleneck: int = 512


# ---------------------------------------------------------------------------
# building blocks (forward and adjoint)
# ---------------------------------------------------------------------------
def conv3(x, w):
    """y[b,o] = sum_i sum_d w[o,i,d] x[b,i,. + d - 1], zero outside."""
    B, _, Z, Y, X = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1), (1, 1)))
    y = np.zeros((B, w.shape[0], Z, Y, X))
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                y += np.einsum("bizyx,oi->bozyx", xp[:, :, dz:dz + Z, dy:dy + Y, dx:dx + X], w[:, :, dz, dy, dx],
                               optimize=True)
    return y


def conv3_backward(x, w, gy):
    """Gradients of conv3 with respect to its input and weights."""
    B, _, Z, Y, X = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1), (1, 1)))
    gxp = np.zeros_like(xp)
    gw = np.zeros_like(w)
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                sl = (slice(None), slice(None), slice(dz, dz + Z), slice(dy, dy + Y), slice(dx, dx + X))
                gw[:, :, dz, dy, dx] = np.einsum("bozyx,bizyx->oi", gy, xp[sl], optimize=True)
                gxp[sl] += np.einsum("bozyx,oi->bizyx", gy, w[:, :, dz, dy, dx], optimize=True)
    return gxp[:, :, 1:-1, 1:-1, 1:-1], gw


def batchnorm(x, gamma, beta):
    """Training-mode batch normalisation over (batch, z, y, x)."""
    mu = x.mean(axis=(0, 2, 3, 4), keepdims=True)
    var = ((x - mu) ** 2).mean(axis=(0, 2, 3, 4), keepdims=True)
    sig = np.sqrt(var + EPS)
    xh = (x - mu) / sig
    return gamma[None, :, None, None, None] * xh + beta[None, :, None, None, None], (xh, sig)


def batchnorm_backward(cache, gamma, gy):
    xh, sig = cache
    ax = (0, 2, 3, 4)
    ggamma = (gy * xh).sum(axis=ax)
    gbeta = gy.sum(axis=ax)
    gxh = gy * gamma[None, :, None, None, None]
    gx = (gxh - gxh.mean(axis=ax, keepdims=True) - xh * (gxh * xh).mean(axis=ax, keepdims=True)) / sig
    return gx, ggamma, gbeta


def maxpool2(x):
    """2x2x2 max-pooling, stride 2; also the index (0..7) of the maximum in
    each window (offsets dz*4 + dy*2 + dx; the first in that order wins)."""
    B, C, Z, Y, X = x.shape
    best = np.full((B, C, Z // 2, Y // 2, X // 2), -np.inf)
    arg = np.zeros(best.shape, dtype=np.int64)
    for k in range(8):
        dz, dy, dx = k >> 2, (k >> 1) & 1, k & 1
        v = x[:, :, dz::2, dy::2, dx::2]
        better = v > best
        best = np.where(better, v, best)
        arg = np.where(better, k, arg)
    return best, arg


def maxpool2_backward(arg, gy, shape):
    gx = np.zeros(shape)
    for k in range(8):
        dz, dy, dx = k >> 2, (k >> 1) & 1, k & 1
        gx[:, :, dz::2, dy::2, dx::2] = np.where(arg == k, gy, 0.0)
    return gx


def upsample_matrix(n):
    """[2n, n] linear map of the cell-centred up-sampling by 2 along one axis."""
    m = np.zeros((2 * n, n))
    for o in range(2 * n):
        s = min(max((o + 0.5) / 2.0 - 0.5, 0.0), n - 1.0)
        i0 = int(np.floor(s))
        i1 = min(i0 + 1, n - 1)
        w = s - i0
        m[o, i0] += 1.0 - w
        m[o, i1] += w
    return m


def up2(x):
    _, _, Z, Y, X = x.shape
    return np.einsum("az,by,cx,nkzyx->nkabc", upsample_matrix(Z), upsample_matrix(Y), upsample_matrix(X), x,
                     optimize=True)


def up2_backward(gy, shape):
    _, _, Z, Y, X = shape
    return np.einsum("az,by,cx,nkabc->nkzyx", upsample_matrix(Z), upsample_matrix(Y), upsample_matrix(X), gy,
                     optimize=True)


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


# ---------------------------------------------------------------------------
# network
# ---------------------------------------------------------------------------
def block_names(cfg):
    """Convolution blocks in forward order: (name, in channels, out channels)."""
    out = []
    cin = cfg.cin
    for e, c in enumerate(cfg.channels):
        out += [(f"enc{e}a", cin, c), (f"enc{e}b", c, c)]
        cin = c
    out += [("mida", cin, cfg.bottleneck), ("midb", cfg.bottleneck, cfg.bottleneck)]
    below = cfg.bottleneck
    for d in reversed(range(len(cfg.channels))):
        c = cfg.channels[d]
        out += [(f"dec{d}a", c + below, c), (f"dec{d}b", c, c)]
        below = c
    return out


def init_params(cfg, seed=0):
    """He-normal convolution weights, gamma = 1, beta = 0, uniform output
    layer (the initialisation is not part of the method; any seeded draw)."""
    r = np.random.Generator(np.random.PCG64(seed))
    p = {}
    for name, ci, co in block_names(cfg):
        p[name + "_w"] = r.normal(size=(co, ci, 3, 3, 3)) * np.sqrt(2.0 / (27 * ci))
        p[name + "_g"] = np.ones(co)
        p[name + "_b"] = np.zeros(co)
    c0 = cfg.channels[0]
    p["out_w"] = r.uniform(-1, 1, size=(cfg.cout, c0)) / np.sqrt(c0)
    p["out_b"] = np.zeros(cfg.cout)
    return p


def _block(p, name, x, tape):
    z = conv3(x, p[name + "_w"])
    n, cache = batchnorm(z, p[name + "_g"], p[name + "_b"])
    y = np.maximum(n, 0.0)
    tape.append((name, x, cache, n))
    return y


def forward(p, x, cfg, keep=False):
    """y = sigmoid(out(decoder(encoder(x)))); with keep, also the tape for
    backward."""
    tape = []
    skips, pools = [], []
    h = x
    for e in range(len(cfg.channels)):
        h = _block(p, f"enc{e}a", h, tape)
        h = _block(p, f"enc{e}b", h, tape)
        skips.append(h)
        h, arg = maxpool2(h)
        pools.append((arg, skips[-1].shape))
    h = _block(p, "mida", h, tape)
    h = _block(p, "midb", h, tape)
    ups = []
    for d in reversed(range(len(cfg.channels))):
        u = up2(h)
        ups.append((h.shape, skips[d].shape[1]))
        h = np.concatenate([skips[d], u], axis=1)
        h = _block(p, f"dec{d}a", h, tape)
        h = _block(p, f"dec{d}b", h, tape)
    a = np.einsum("oc,bczyx->bozyx", p["out_w"], h, optimize=True) + p["out_b"][None, :, None, None, None]
    y = sigmoid(a)
    if keep:
        return y, dict(blocks=tape, pools=pools, ups=ups, last=h)
    return y


def _block_backward(p, entry, gy, g):
    name, x, cache, n = entry
    gn = gy * (n > 0)
    gz, g[name + "_g"], g[name + "_b"] = batchnorm_backward(cache, p[name + "_g"], gn)
    gx, g[name + "_w"] = conv3_backward(x, p[name + "_w"], gz)
    return gx


def backward(p, tape, y, t, m, cfg):
    """Gradients of masked_mse(y, t, m) with respect to every parameter."""
    g = {}
    C = y.shape[1]
    gy = 2.0 * m[:, None] * (y - t) / (C * m.sum())
    ga = gy * y * (1.0 - y)
    h = tape["last"]
    g["out_w"] = np.einsum("bozyx,bczyx->oc", ga, h, optimize=True)
    g["out_b"] = ga.sum(axis=(0, 2, 3, 4))
    gh = np.einsum("oc,bozyx->bczyx", p["out_w"], ga, optimize=True)
    blocks = list(tape["blocks"])
    nd = len(cfg.channels)
    gskip = [None] * nd
    ups = tape["ups"]
    for j, d in enumerate(range(nd)):                 # decoder, last stage first
        gh = _block_backward(p, blocks.pop(), gh, g)
        gh = _block_backward(p, blocks.pop(), gh, g)
        below_shape, cs = ups[nd - 1 - j]
        gskip[d] = gh[:, :cs]
        gh = up2_backward(gh[:, cs:], below_shape)
    gh = _block_backward(p, blocks.pop(), gh, g)      # bottleneck
    gh = _block_backward(p, blocks.pop(), gh, g)
    for e in reversed(range(nd)):                      # encoder
        arg, shape = tape["pools"][e]
        gh = maxpool2_backward(arg, gh, shape) + gskip[e]
        gh = _block_backward(p, blocks.pop(), gh, g)
        gh = _block_backward(p, blocks.pop(), gh, g)
    g["input"] = gh
    return g


masked_mse = _fno.masked_mse
adam_step = _fno.adam_step


def loss_and_grad(p, x, t, m, cfg):
    y, tape = forward(p, x, cfg, keep=True)
    return masked_mse(y, t, m), backward(p, tape, y, t, m, cfg)


def macs(cfg):
    """Multiply-accumulates of one forward pass of one sample (convolutions
    and the output layer)."""
    nz, ny, nx = cfg.grid
    total, cells = 0, nz * ny * nx
    ch = [cfg.cin] + list(cfg.channels)
    for e, c in enumerate(cfg.channels):
        total += cells * 27 * (ch[e] * c + c * c)
        cells //= 8
    total += cells * 27 * (cfg.channels[-1] * cfg.bottleneck + cfg.bottleneck ** 2)
    below = cfg.bottleneck
    for d in reversed(range(len(cfg.channels))):
        cells *= 8
        c = cfg.channels[d]
        total += cells * 27 * ((c + below) * c + c * c)
        below = c
    total += cells * cfg.channels[0] * cfg.cout
    return total
