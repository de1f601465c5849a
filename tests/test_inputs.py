"""Seeded input generators: SplitMix64 against its published outputs,
deterministic masks with the expected geometry."""
import os

import numpy as np

from paper_2606_16765_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_seed0.txt")


def test_splitmix64_reference_outputs():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    for ctr, hexval in rows:
        assert int(I.splitmix64(0, int(ctr))) == int(hexval, 16)


def test_splitmix64_vectorised_matches_scalar_bigint():
    M = (1 << 64) - 1

    def ref(seed, k):
        z = (seed + (k + 1) * 0x9E3779B97F4A7C15) & M
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        return z ^ (z >> 31)

    ks = np.array([0, 1, 2, 12345, 2**40 + 7, 2**63 - 5], dtype=np.uint64)
    got = I.splitmix64(987654321, ks)
    for k, g in zip(ks, got):
        assert int(g) == ref(987654321, int(k))
    u = I.uniform_pm1(3, np.arange(100000))
    assert u.min() >= -1 and u.max() < 1 and abs(u.mean()) < 0.01


def test_sphere_mask_volume_and_symmetry():
    m = I.sphere((64, 32, 32), (16.0, 15.5, 15.5), 4.0)
    assert m.dtype == np.uint8 and m.shape == (32, 32, 64)
    assert abs(int(m.sum()) - 4 / 3 * np.pi * 4 ** 3) < 0.1 * 268
    assert np.array_equal(m, m[:, ::-1, :]) and np.array_equal(m, m[::-1, :, :])
    assert np.array_equal(m, m.transpose(1, 0, 2))


def test_cylinder_spans_the_channel():
    m = I.cylinder_z((256, 128, 128), (64.0, 63.5), 16.0)
    assert np.all(m.sum(axis=0)[m[0] > 0] == 128)
    area = m[0].sum()
    assert abs(area - np.pi * 64) < 0.1 * np.pi * 64


def test_composite_obstacle_is_deterministic_and_placed():
    a = I.composite(7, (256, 128, 128), size_range=(10, 30))
    b = I.composite(7, (256, 128, 128), size_range=(10, 30))
    ma, mb = a.mask(), b.mask()
    assert np.array_equal(ma, mb) and ma.sum() > 0
    assert 2 <= len(a.prims) <= 4 and -30 <= a.angle_deg <= 30
    z, y, x = np.nonzero(ma)
    assert abs(x.mean() - 0.3 * 256) < 25
    c = I.composite(8, (256, 128, 128), size_range=(10, 30)).mask()
    assert not np.array_equal(ma, c)
    for kind in I.PRIMITIVES:
        p = I.Primitive(kind, (40.0, 30.0, 30.0), (20.0, 12.0, 16.0), 10.0)
        assert I.voxelize((80, 60, 60), [p]).sum() > 50, kind


def test_batch_channels_shapes():
    b = I.batch_channels(0, n=6)
    for d in b:
        nx, ny, nz = d["grid"]
        assert nx in (128, 192, 256) and ny in (64, 96, 128) and nz in (64, 96, 128)
        assert 1000 <= d["re"] <= 10000
        assert d["mask"].shape == (nz, ny, nx) and d["mask"].sum() > 0


def test_link_wall_distances_match_the_sphere_intersection():
    """Bisection wall distances of the fluid-to-obstacle links against the
    closed-form intersection of each link segment with the sphere."""
    g = (20, 16, 16)
    C, R = np.array([9.3, 7.6, 8.1]), 3.5
    cell, d, q = I.link_wall_distances(g, [I.Primitive("sphere", tuple(C), (2 * R,))])
    m = I.sphere(g, tuple(C), R)
    nx, ny = g[0], g[1]
    X, Y, Z = cell % nx, (cell // nx) % ny, cell // (nx * ny)
    cv = np.array([[j % 3 - 1, (j // 3) % 3 - 1, j // 9 - 1] for j in range(27)], float)
    V = cv[d.astype(int)]
    P = np.stack([X, Y, Z], 1).astype(float)
    assert (m.reshape(-1)[cell] == 0).all()
    tgt = P + V
    assert (m[tgt[:, 2].astype(int), tgt[:, 1].astype(int), tgt[:, 0].astype(int)] == 1).all()
    a, b, c = (V * V).sum(1), 2 * ((P - C) * V).sum(1), ((P - C) ** 2).sum(1) - R * R
    s = (-b - np.sqrt(b * b - 4 * a * c)) / (2 * a)
    assert np.abs(s - q).max() < 1e-10
    # every fluid-to-solid link is listed once
    n_links = 0
    for j in range(27):
        if j == 13:
            continue
        sh = np.roll(np.roll(np.roll(m, -int(cv[j, 2]), 0), -int(cv[j, 1]), 1), -int(cv[j, 0]), 2)
        n_links += int(((m == 0) & (sh == 1)).sum())
    assert len(cell) == n_links
