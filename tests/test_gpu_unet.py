"""The U-Net on the GPU (libunet.so: tcgen05 implicit-GEMM convolutions, BF16
activations) against the FP64 oracle (oracle/unet.py).

The convolutions alone are compared exactly up to FP32 summation: their
inputs and weights are drawn as BF16 values, so the tensor cores' products
are exact and only the FP32 sums differ from the oracle.  The rounding error
of a sum of K such products grows as sqrt(K) 2^-24 of its magnitude (the
roundings act as independent errors of random sign), so the bound is
4 sqrt(K) 2^-24 of the largest output, K the contraction length.

The network stores every activation in BF16 (each convolution output, each
normalised output and each up-sampled field are rounded, about 2^-9
relative).  Max-pooling and ReLU turn such roundings into discrete changes
(a different maximum of a window, a flipped sign), so on small grids the
gradients of the early layers move by tens of percent between the FP64 and
a BF16-stored network.  The network tests therefore compare the GPU with
the oracle evaluated with the same BF16 storage points (`_rounded`), and
check that the GPU is no further from the exact FP64 oracle than that
rounded oracle is."""
import contextlib
import math
import numpy as np
import pytest

import oracle.unet as U

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def bf16(a):
    """Round to the nearest BF16 value (ties to even), returned as float32."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _conv_case(seed, B, nz, ny, nx, cin, cout):
    r = np.random.default_rng(seed)
    x = bf16(r.normal(size=(B, nz, ny, nx, cin)))
    w = bf16(r.normal(size=(cout, cin, 27)) / np.sqrt(27 * cin))
    g = bf16(r.normal(size=(B, nz, ny, nx, cout)))
    return x, w, g


def _sum_tol(K):
    """Bound on the largest error of K-term FP32 sums of exact products,
    relative to the largest output (see the module docstring)."""
    return 4.0 * math.sqrt(K) * 2.0 ** -24


@contextlib.contextmanager
def _rounded():
    """The oracle with the GPU's BF16 storage points: convolution outputs,
    normalised outputs and up-sampled fields rounded to BF16 (round to
    nearest even); the backward stays the oracle's exact FP64 adjoint of
    that forward."""
    block, up2 = U._block, U.up2

    def rblock(p, name, x, tape):
        z = bf16(U.conv3(x, p[name + "_w"])).astype(np.float64)
        n, cache = U.batchnorm(z, p[name + "_g"], p[name + "_b"])
        tape.append((name, x, cache, n))
        return bf16(np.maximum(n, 0.0)).astype(np.float64)

    U._block = rblock
    U.up2 = lambda x: bf16(up2(x)).astype(np.float64)
    try:
        yield
    finally:
        U._block, U.up2 = block, up2


def _rel(a, b):
    a, b = np.ravel(a), np.ravel(b)
    return float(np.linalg.norm(a - b) / (np.linalg.norm(b) + 1e-300))


def _cos(a, b):
    a, b = np.ravel(a), np.ravel(b)
    return float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-300))


def _first(a):
    """[B, z, y, x, C] -> [B, C, z, y, x] float64"""
    return np.moveaxis(a.astype(np.float64), -1, 1)


def _w5(w):
    return w.astype(np.float64).reshape(w.shape[0], w.shape[1], 3, 3, 3)


# grids: a 128-cell row tile; tiles spanning rows, planes and samples (with
# the last tile past the batch); 64- and 32-channel chunks; N split in tiles
CONV_CASES = [
    (2, 8, 8, 16, 64, 96),
    (3, 2, 4, 4, 32, 32),
    (2, 4, 4, 8, 96, 384),
    (1, 4, 8, 128, 32, 64),
]


@pytest.mark.parametrize("case", CONV_CASES)
def test_conv3_forward_matches_fp64(case):
    _need_gpu()
    from paper_2606_16765_gb300 import unet as N
    B, nz, ny, nx, cin, cout = case
    x, w, _ = _conv_case(1, B, nz, ny, nx, cin, cout)
    y = torch.zeros((B, nz, ny, nx, cout), device="cuda")
    N.conv3_forward(_dev(x), _dev(w), y)
    ref = np.moveaxis(U.conv3(_first(x), _w5(w)), 1, -1)
    err = np.abs(y.cpu().numpy() - ref).max() / np.abs(ref).max()
    tol = _sum_tol(27 * cin)
    print(f"conv3 forward {case}: max rel err {err:.2e} (bound {tol:.2e})")
    assert err < tol


@pytest.mark.parametrize("case", CONV_CASES)
def test_conv3_backward_matches_fp64(case):
    _need_gpu()
    from paper_2606_16765_gb300 import unet as N
    B, nz, ny, nx, cin, cout = case
    x, w, g = _conv_case(2, B, nz, ny, nx, cin, cout)
    gx = torch.zeros((B, nz, ny, nx, cin), device="cuda")
    gw = torch.zeros((cout, cin, 27), device="cuda")
    N.conv3_backward_data(_dev(g), _dev(w), gx)
    N.conv3_backward_weights(_dev(x), _dev(g), gw)
    rgx, rgw = U.conv3_backward(_first(x), _w5(w), _first(g))
    rgx = np.moveaxis(rgx, 1, -1)
    rgw = rgw.reshape(cout, cin, 27)
    ex = np.abs(gx.cpu().numpy() - rgx).max() / np.abs(rgx).max()
    ew = np.abs(gw.cpu().numpy() - rgw).max() / np.abs(rgw).max()
    tx, tw = _sum_tol(27 * cout), _sum_tol(B * nz * ny * nx)
    print(f"conv3 backward {case}: input gradient {ex:.2e} (bound {tx:.2e}), weight gradient {ew:.2e} "
          f"(bound {tw:.2e})")
    assert ex < tx and ew < tw


def _net_case(B=2, grid=(16, 16, 32), stages=3, channels=(32, 64, 128), bottleneck=128, seed=3):
    cfg = U.UNetConfig(grid=grid, cin=4, cout=4, channels=channels, bottleneck=bottleneck)
    r = np.random.default_rng(seed)
    nz, ny, nx = grid
    x = np.zeros((B, 4) + grid)
    x[:, 0] = (r.uniform(size=(B,) + grid) < 0.2)             # an obstacle-like binary channel
    x[:, 1] = r.uniform(-0.5, 0.5, size=(B, 1, 1, 1))          # log10 Re - 3.5
    ang = r.uniform(-0.5, 0.5, size=B)
    x[:, 2] = np.cos(ang)[:, None, None, None]
    x[:, 3] = np.sin(ang)[:, None, None, None]
    x = bf16(x).astype(np.float64)
    t = r.uniform(0.2, 0.8, size=(B, 4) + grid)
    m = (r.uniform(size=(B,) + grid) < 0.8).astype(np.float64)
    p = U.init_params(cfg, seed=seed + 1)
    for k in p:
        if k.endswith("_w") and k != "out_w":
            p[k] = bf16(p[k]).astype(np.float64)                # the GPU stores BF16 weights
        if k.endswith("_g"):
            p[k] = 1.0 + 0.2 * r.normal(size=p[k].shape)
        if k.endswith("_b") and k != "out_b":
            p[k] = 0.1 * r.normal(size=p[k].shape)
    kw = dict(nx=nx, ny=ny, nz=nz, cin=4, cout=4, stages=stages, channels=channels, bottleneck=bottleneck,
              max_batch=B)
    return cfg, kw, x, t, m, p


def _gpu_net(kw, cfg, p):
    from paper_2606_16765_gb300 import unet as N
    net = N.UNet(**kw)
    assert [(n, ci, co) for n, ci, co in N.blocks(net.cfg)] == U.block_names(cfg)
    net.set_params(N.flatten(net.cfg, p))
    return net


def test_forward_matches_oracle():
    _need_gpu()
    cfg, kw, x, t, m, p = _net_case()
    net = _gpu_net(kw, cfg, p)
    y = net.forward(x.astype(np.float32))
    net.sync()
    net.close()
    _check_forward(y, p, x, cfg, "U-Net forward")


def _check_forward(y, p, x, cfg, label):
    """The GPU output against the BF16-stored oracle (tight) and against the
    exact oracle (no further than the BF16-stored oracle is)."""
    ref = U.forward(p, x, cfg)
    with _rounded():
        rnd = U.forward(p, x, cfg)
    scale = np.linalg.norm(ref - ref.mean())
    e_gpu_rnd = np.linalg.norm(y - rnd) / scale
    e_gpu_ref = np.linalg.norm(y - ref) / scale
    e_rnd_ref = np.linalg.norm(rnd - ref) / scale
    print(f"{label}: rel L2 about the mean: GPU vs BF16-stored oracle {e_gpu_rnd:.2e}, GPU vs FP64 oracle "
          f"{e_gpu_ref:.2e}, BF16-stored vs FP64 oracle {e_rnd_ref:.2e}")
    # the GPU shares the storage points: it sits closer to the BF16-stored
    # oracle than that is to the exact one, and no further from the exact
    # oracle than BF16 storage itself moves it
    assert e_gpu_rnd < e_rnd_ref + 2e-3
    assert e_gpu_ref < 1.5 * e_rnd_ref + 2e-3


def test_gradients_match_oracle():
    _need_gpu()
    from paper_2606_16765_gb300 import unet as N
    cfg, kw, x, t, m, p = _net_case()
    net = _gpu_net(kw, cfg, p)
    L = net.loss_grad(x.astype(np.float32), t.astype(np.float32), m.astype(np.float32))
    net.sync()
    g = N.unflatten(net.cfg, net.grads())
    net.close()
    Lr, gr = U.loss_and_grad(p, x, t, m, cfg)
    with _rounded():
        Ls, gs = U.loss_and_grad(p, x, t, m, cfg)
    assert abs(L - Lr) < 1e-3 * Lr and abs(L - Ls) < 1e-3 * Ls
    worst = []
    for k in gr:
        if k == "input":
            continue
        worst.append((_rel(g[k], gs[k]), _cos(g[k], gs[k]), _rel(g[k], gr[k]), _rel(gs[k], gr[k]), k))
    worst.sort(reverse=True)
    print("U-Net gradients, worst groups (rel L2 and cosine vs the BF16-stored oracle; rel L2 of the GPU and of the "
          "BF16-stored oracle vs the FP64 oracle):",
          [(f"{a:.2e}", f"{c:.5f}", f"{e:.2e}", f"{r:.2e}", k) for a, c, e, r, k in worst[:6]])
    for rel, cos, e_ref, r_ref, k in worst:
        # the GPU's backward also rounds the gradients to BF16 (a smooth
        # perturbation of a few 2^-9 over the blocks) on top of the forward's
        # storage effects, which the BF16-stored oracle shares
        assert rel < r_ref + 0.03, (k, rel, r_ref)
        assert e_ref < 1.5 * r_ref + 0.03, (k, e_ref, r_ref)


def test_adam_steps_follow_the_oracle():
    _need_gpu()
    cfg, kw, x, t, m, p = _net_case(seed=7)
    net = _gpu_net(kw, cfg, p)
    pr = {k: v.copy() for k, v in p.items()}
    m1 = {k: np.zeros_like(v) for k, v in p.items()}
    m2 = {k: np.zeros_like(v) for k, v in p.items()}
    lg, lr_ = [], []
    for step in range(1, 6):
        lg.append(net.train_step(x.astype(np.float32), t.astype(np.float32), m.astype(np.float32), 1e-3))
        L, g = U.loss_and_grad(pr, x, t, m, cfg)
        g.pop("input")
        lr_.append(L)
        U.adam_step(pr, g, m1, m2, step, 1e-3)
    net.sync()
    print("U-Net Adam losses GPU", [f"{v:.5f}" for v in lg], "oracle", [f"{v:.5f}" for v in lr_])
    net.close()
    assert lg[-1] < lg[0] and lr_[-1] < lr_[0]
    for a, b in zip(lg, lr_):
        assert abs(a - b) < 0.02 * b


def test_full_size_forward_matches_oracle():
    """The paper's configuration (128x64x64, encoder [32, 64, 128, 256],
    bottleneck 512) at batch 1 against the oracle."""
    _need_gpu()
    cfg, kw, x, t, m, p = _net_case(B=1, grid=(64, 64, 128), stages=4, channels=(32, 64, 128, 256), bottleneck=512,
                                    seed=11)
    net = _gpu_net(kw, cfg, p)
    y = net.forward(x.astype(np.float32))
    net.sync()
    net.close()
    _check_forward(y, p, x, cfg, "U-Net 128x64x64 forward")


def test_timed_training_step_paper_configuration():
    """Batch 8 on 128x64x64: a training step's time (CUDA events) and a loss
    that falls over a few steps on fixed synthetic data."""
    _need_gpu()
    from paper_2606_16765_gb300 import unet as N
    net = N.UNet()
    B = 8
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.rand((B, 4, 64, 64, 128), device="cuda", generator=g)
    x[:, 0] = (x[:, 0] < 0.1).float()
    t = torch.rand((B, 4, 64, 64, 128), device="cuda", generator=g) * 0.5 + 0.25
    m = torch.ones((B, 64, 64, 128), device="cuda")
    losses = [net.train_step(x, t, m, 1e-3) for _ in range(3)]
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(5):
        losses.append(net.train_step(x, t, m, 1e-3))
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 5
    e0.record(st)
    y = torch.empty_like(t)
    for _ in range(5):
        net.forward(x, y)
    e1.record(st)
    torch.cuda.synchronize()
    fms = e0.elapsed_time(e1) / 5
    net.sync()
    net.close()
    print(f"U-Net batch 8: training step {ms:.2f} ms ({B / ms * 1e3:.1f} samples/s), forward {fms:.2f} ms; "
          f"losses {[round(v, 5) for v in losses]}")
    assert losses[-1] < losses[0]
