"""Host side of the sphere validation runs (Table 1): the stored table, the
geometry of the validation channel and the drag normalisation."""
import math
import os

import numpy as np
import pytest

from paper_2606_16765_gb300 import sphere_validation as V

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_sphere_drag.txt")


def read_table1():
    cols = [128, 256, 384, 512, 1024]
    out = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        re_s, re_c = int(f[0]), int(f[1])
        assert re_c == 6 * re_s                          # D = L/6
        out[re_s] = {L: float(v) for L, v in zip(cols, f[2:7]) if v != "-"}
    return out


def test_module_table_is_the_printed_table():
    assert V.TABLE1 == read_table1()


@pytest.mark.parametrize("L", [128, 256])
def test_validation_channel_geometry(L):
    grid, D, c, prims, mask, (cell, d, q) = V.sphere_channel(L)
    assert grid == (2 * L, L, L) and D == pytest.approx(L / 6)
    assert c[0] / (2 * L) == pytest.approx(0.3)          # x / 2L = 0.3, centred in y and z
    # the voxel volume approaches the sphere's (cell centres inside)
    assert mask.sum() == pytest.approx(math.pi * D ** 3 / 6, rel=0.03)
    # one link per (fluid cell, direction into the sphere), wall distance in (0, 1)
    assert len(cell) == len(d) == len(q) > 0 and (q > 0).all() and (q < 1).all()
    nx, ny, _ = grid
    x, y, z = cell % nx, (cell // nx) % ny, cell // (nx * ny)
    assert (mask[z, y, x] == 0).all()
    cx, cy, cz = d % 3 - 1, (d // 3) % 3 - 1, d // 9 - 1
    assert (mask[z + cz, y + cy, x + cx] == 1).all()
    # the crossing point lies on the sphere
    p = np.stack([x + q * cx, y + q * cy, z + q * cz], 1) - np.array(c)
    assert np.abs(np.linalg.norm(p, axis=1) - D / 2).max() < 1e-9


def test_drag_normalisation():
    D = 128 / 6
    fx = np.full(50, 0.5 * V.U ** 2 * math.pi * D * D / 4 * 1.1)
    assert V.drag_coefficient(fx, D) == pytest.approx(1.1)


def test_centreline_is_the_mean_of_the_four_rows_around_the_axis():
    f = np.zeros((4, 6, 5))
    f[1, 2], f[1, 3], f[2, 2], f[2, 3] = 1.0, 2.0, 3.0, 6.0
    assert np.allclose(V.centreline(f, (0.0, 2.5, 1.5)), 3.0)
    g = np.arange(4 * 6 * 5, dtype=float).reshape(4, 6, 5)
    assert np.allclose(V.centreline(g, (0.0, 3.0, 2.0)), g[2, 3])      # on a cell centre: that row


def test_profile_peaks_of_a_two_bump_profile():
    xs = np.linspace(0.0, 6.0, 601)
    v = np.exp(-((xs - 1.5) / 0.2) ** 2) + 1.2 * np.exp(-((xs - 2.4) / 0.3) ** 2) + 0.3 * np.exp(-((xs - 4.0) / 0.2) ** 2)
    assert V.profile_peaks(v, xs, 0.5, 5.0) == pytest.approx([1.5, 2.4], abs=0.02)
    assert V.profile_peaks(v, xs, 0.5, 5.0, count=3)[-1] == pytest.approx(4.0, abs=0.02)
    assert V.profile_peaks(v, xs, 2.0, 5.0, count=1) == pytest.approx([2.4], abs=0.02)
