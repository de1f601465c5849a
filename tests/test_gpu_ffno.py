"""The factorised FNO on the GPU (libffno.so, FP32) against the FP64 oracle
(oracle/ffno.py): forward, loss, every gradient group, and an Adam
trajectory, on a tiny network and on a grid of several blocks per row."""
import numpy as np
import pytest

from oracle import ffno as F

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


CASES = {
    "tiny": dict(grid=(6, 5, 8), cin=2, width=3, cout=2, modes=(2, 3, 4), layers=2, ff_hidden=4, hidden=5,
                 lift_hidden=3, B=2),
    "rows": dict(grid=(8, 16, 32), cin=4, width=8, cout=4, modes=(3, 5, 9), layers=2, ff_hidden=8, hidden=16,
                 lift_hidden=8, B=3),
}


def _setup(name, seed):
    from paper_2606_16765_gb300 import ffno as G
    kw = dict(CASES[name])
    B = kw.pop("B")
    cfg = F.FFNOConfig(**kw)
    nz, ny, nx = cfg.grid
    mz, my, mx = cfg.modes
    net = G.FFNO(nx=nx, ny=ny, nz=nz, cin=cfg.cin, width=cfg.width, cout=cfg.cout, mx=mx, my=my, mz=mz,
                 layers=cfg.layers, ff_hidden=cfg.ff_hidden, hidden=cfg.hidden, lift_hidden=cfg.lift_hidden,
                 max_batch=B)
    p = F.init_params(cfg, seed=seed)
    net.set_params(G.flatten(net.cfg, p))
    r = np.random.default_rng(seed + 100)
    x = r.normal(size=(B, cfg.cin) + cfg.grid).astype(np.float32)
    t = r.normal(size=(B, cfg.cout) + cfg.grid).astype(np.float32)
    m = (r.uniform(size=(B,) + cfg.grid) < 0.7).astype(np.float32)
    return G, cfg, net, p, x, t, m


@pytest.mark.parametrize("name", list(CASES))
def test_forward_loss_and_gradients_match_oracle(name):
    _need_gpu()
    G, cfg, net, p, x, t, m = _setup(name, 1)
    y = net.forward(x)
    yr = F.forward(p, x.astype(np.float64), cfg)
    ferr = np.abs(y - yr).max() / np.abs(yr).max()
    L = net.loss_grad(x, t, m)
    Lr, gr = F.loss_and_grad(p, x.astype(np.float64), t.astype(np.float64), m.astype(np.float64), cfg)
    g = G.unflatten(net.cfg, net.grads())
    worst = max(np.linalg.norm((g[k] - gr[k]).ravel()) / (np.linalg.norm(gr[k].ravel()) + 1e-300) for k in g)
    print(f"FFNO {name}: forward {ferr:.2e}, loss {abs(L - Lr) / Lr:.2e}, worst gradient group {worst:.2e}")
    net.close()
    assert ferr < 1e-5 and abs(L - Lr) < 1e-6 * Lr and worst < 1e-4


def test_adam_trajectory_matches_oracle():
    """Three Adam steps: the losses along the way, and each group's
    displacement (an Adam step is about the learning rate per entry whatever
    the gradient's size, so entries whose gradient is at rounding level may
    differ; the groups' displacements as a whole must agree)."""
    _need_gpu()
    G, cfg, net, p, x, t, m = _setup("tiny", 2)
    pr = {k: v.copy() for k, v in p.items()}
    m1 = {k: np.zeros_like(v) for k, v in p.items()}
    m2 = {k: np.zeros_like(v) for k, v in p.items()}
    lg, lr_ = [], []
    for step in range(1, 4):
        lg.append(net.loss_grad(x, t, m))
        net.adam(1e-3)
        L, g = F.loss_and_grad(pr, x.astype(np.float64), t.astype(np.float64), m.astype(np.float64), cfg)
        lr_.append(L)
        g.pop("input")
        F.adam_step(pr, g, m1, m2, step, 1e-3)
    q = G.unflatten(net.cfg, net.params())
    net.close()
    for a, b in zip(lg, lr_):
        assert abs(a - b) < 1e-5 * b
    for k in q:
        dg, dr = (q[k] - p[k]).ravel(), (pr[k] - p[k]).ravel()
        cos = float(np.real(np.vdot(dg, dr)) / (np.linalg.norm(dg) * np.linalg.norm(dr) + 1e-300))
        rel = float(np.linalg.norm(dg - dr) / (np.linalg.norm(dr) + 1e-300))
        assert cos > 0.999 and rel < 1e-2, (k, cos, rel)
