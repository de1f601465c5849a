"""Host side of the FNO data / evaluation pipeline: seeded samples, input
features, loss-region weights and the evaluation metrics against closed
forms."""
import math

import numpy as np
import pytest

from paper_2606_16765_gb300 import fno_pipeline as P


def test_samples_are_deterministic_and_in_range():
    a, b = P.sample(3), P.sample(3)
    assert a["re"] == b["re"] and np.array_equal(a["mask"], b["mask"]) and a["angle"] == b["angle"]
    ss = [P.sample(s) for s in range(40)]
    res = [s["re"] for s in ss]
    assert min(res) >= P.RE_RANGE[0] and max(res) <= P.RE_RANGE[1] == 10000.0 and P.RE_RANGE[0] == 1000.0
    # the batched configuration's grids, each axis from its set, several of them drawn
    grids = {s["grid"] for s in ss}
    assert len(grids) > 5
    for g in grids:
        assert g[0] in (128, 192, 256) and g[1] in (64, 96, 128) and g[2] in (64, 96, 128)
    for s in ss[:6]:
        m = s["mask"]
        assert m.shape == (s["grid"][2], s["grid"][1], s["grid"][0]) and 0 < m.sum() < m.size
        assert -30.0 <= s["angle"] <= 30.0
    d = P.sample(3, grids="direct")
    assert d["grid"] == P.GRID and d["mask"].shape == (P.GRID[2], P.GRID[1], P.GRID[0])


def test_target_mask_samples_the_geometry_on_the_surrogate_grid():
    """On the surrogate's own grid the target mask is the voxelised mask; on
    a grid twice as fine along every axis it agrees with the fine mask on
    every 2x2x2 block that is wholly fluid or wholly solid."""
    d = P.sample(4, grids="direct")
    assert np.array_equal(P.target_mask(d), d["mask"])
    s = next(P.sample(k) for k in range(100) if P.sample(k)["grid"] == (256, 128, 128))
    m = P.target_mask(s)
    assert m.shape == (P.GRID[2], P.GRID[1], P.GRID[0])
    fine = s["mask"].astype(np.float64)
    box = fine.reshape(64, 2, 64, 2, 128, 2).mean(axis=(1, 3, 5))
    clear = (box == 0) | (box == 1)                      # blocks entirely fluid or solid
    assert np.array_equal(m[clear], box[clear].astype(np.uint8))
    assert m.sum() > 0


def test_features_channels():
    s = P.sample(5)
    f = P.features(s)
    assert f.shape == (4, P.GRID[2], P.GRID[1], P.GRID[0])
    assert np.array_equal(f[0], P.target_mask(s).astype(np.float32))
    centre = 0.5 * (math.log10(P.RE_RANGE[0]) + math.log10(P.RE_RANGE[1]))
    assert centre == pytest.approx(3.5)
    assert np.allclose(f[1], math.log10(s["re"]) - centre)
    a = math.radians(s["angle"])
    assert np.allclose(f[2], math.cos(a)) and np.allclose(f[3], math.sin(a))
    # the geometric mean of the range maps to 0
    s2 = dict(s, re=math.sqrt(P.RE_RANGE[0] * P.RE_RANGE[1]))
    assert np.allclose(P.features(s2)[1], 0.0, atol=1e-6)


def test_region_weights_cover_the_inner_box_fluid_cells():
    nz, ny, nx = 64, 64, 128
    mask = np.zeros((nz, ny, nx), np.uint8)
    mask[30:34, 30:34, 40:44] = 1
    w = P.region_weights(mask)
    x0, x1 = int(0.1 * nx), int(0.9 * nx)          # cells [12, 115) along x
    assert w.sum() == 32 * 32 * (x1 - x0) - 4 * 4 * 4
    assert w[0].sum() == 0 and w[:, :, :x0].sum() == 0 and w[:, :, x1:].sum() == 0
    assert np.all(w[mask == 1] == 0)


def test_metrics_closed_forms():
    r = np.random.default_rng(0)
    true = r.normal(size=(2, 4, 4, 5, 6))
    cells = np.ones((2, 4, 5, 6), bool)
    cells[1, 0] = False
    eps = 0.03
    pred = true.copy()
    pred[:, :3] *= 1 + eps
    pred[:, 3] += 7.0                          # a pressure offset is not an error
    rel, per = P.metrics(pred, true, cells)
    assert rel == pytest.approx([eps, eps])
    for k in ("u", "v", "w"):
        assert per[k] == pytest.approx([eps, eps])
    assert per["p"] == pytest.approx([0.0, 0.0], abs=1e-12)
