"""Seeded synthetic inputs shared by the CUDA path and the FP64 oracle.

This module holds no lattice Boltzmann arithmetic: it only builds obstacle
masks (Sec. 2 of the paper: derived objects from the primitives Cylinder,
Rectangle, Sphere, Torus and Wedge; Sec. 3.1: object at x/2L = 0.3, centred in
the y-z plane, varying angle of attack) and counter-based random numbers.

Conventions: grids are (nx, ny, nz) with x streamwise; masks are uint8 arrays
of shape [nz, ny, nx], 1 = solid; a cell is solid iff its centre (integer
coordinates) lies inside the body.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

PRIMITIVES = ("cylinder", "rectangle", "sphere", "torus", "wedge")

# ---------------------------------------------------------------------------
# counter-based generator: SplitMix64 (Steele, Lea & Flood 2014; the mixing
# constants of Vigna's public-domain reference version)
# ---------------------------------------------------------------------------
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, counter) -> np.ndarray:
    """Output number ``counter`` (0-based) of a SplitMix64 stream started at
    state ``seed``: mix(seed + (counter + 1) * golden)."""
    c = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (c + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniform_pm1(seed: int, counter) -> np.ndarray:
    """Uniform deviates in [-1, 1): 53 high bits of SplitMix64 scaled to
    [0, 1), then 2u - 1 (exact in binary64)."""
    z = splitmix64(seed, counter)
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return 2.0 * u - 1.0


def pdf_noise(seed: int, cells, q: int = 27) -> np.ndarray:
    """Deviates r[i, cell] for the given global cell indices; stream counter
    = cell * q + i."""
    cells = np.asarray(cells, dtype=np.uint64).reshape(-1)
    i = np.arange(q, dtype=np.uint64)
    ctr = cells[None, :] * np.uint64(q) + i[:, None]
    return uniform_pm1(seed, ctr)


# ---------------------------------------------------------------------------
# primitive bodies
# ---------------------------------------------------------------------------
@dataclass
class Primitive:
    kind: str
    center: tuple            # (x, y, z) in cells
    size: tuple              # kind-dependent extents in cells
    angle_deg: float = 0.0   # rotation about the z axis (angle of attack)

    def bbox(self):
        r = 0.5 * math.sqrt(sum(s * s for s in self.size)) + 1.0
        return [(c - r, c + r) for c in self.center]

    def inside(self, X, Y, Z):
        """Inside test at points (cell centres) in grid coordinates."""
        a = math.radians(self.angle_deg)
        dx, dy, dz = X - self.center[0], Y - self.center[1], Z - self.center[2]
        # body frame: rotate the point by -angle about z
        px = math.cos(a) * dx + math.sin(a) * dy
        py = -math.sin(a) * dx + math.cos(a) * dy
        pz = dz
        s = self.size
        if self.kind == "sphere":
            r = 0.5 * s[0]
            return px * px + py * py + pz * pz < r * r
        if self.kind == "cylinder":           # axis along z, diameter s0, length s1
            r = 0.5 * s[0]
            return (px * px + py * py < r * r) & (np.abs(pz) <= 0.5 * s[1])
        if self.kind == "rectangle":          # box with edges s0, s1, s2
            return (np.abs(px) <= 0.5 * s[0]) & (np.abs(py) <= 0.5 * s[1]) & (np.abs(pz) <= 0.5 * s[2])
        if self.kind == "torus":              # ring in the y-z plane (axis x): outer diameter s0, tube diameter s1
            rt = 0.5 * s[1]
            R = 0.5 * s[0] - rt
            q = np.sqrt(py * py + pz * pz) - R
            return q * q + px * px < rt * rt
        if self.kind == "wedge":              # triangular prism: chord s0 (x), height s1 (y), depth s2 (z); apex upstream
            L, H = s[0], s[1]
            t = (px + 0.5 * L) / L            # 0 at the apex, 1 at the base
            return (t >= 0) & (t <= 1) & (np.abs(py) <= 0.5 * H * t) & (np.abs(pz) <= 0.5 * s[2])
        raise ValueError(self.kind)


def voxelize(grid, prims, out=None) -> np.ndarray:
    """Union of primitives on an (nx, ny, nz) grid -> uint8 mask [nz, ny, nx].
    Only each primitive's bounding box is evaluated."""
    nx, ny, nz = grid
    m = np.zeros((nz, ny, nx), np.uint8) if out is None else out
    for p in prims:
        (x0, x1), (y0, y1), (z0, z1) = p.bbox()
        xs = np.arange(max(0, int(math.floor(x0))), min(nx, int(math.ceil(x1)) + 1))
        ys = np.arange(max(0, int(math.floor(y0))), min(ny, int(math.ceil(y1)) + 1))
        zs = np.arange(max(0, int(math.floor(z0))), min(nz, int(math.ceil(z1)) + 1))
        if len(xs) == 0 or len(ys) == 0 or len(zs) == 0:
            continue
        Z, Y, X = np.meshgrid(zs.astype(np.float64), ys.astype(np.float64),
                              xs.astype(np.float64), indexing="ij")
        ins = p.inside(X, Y, Z)
        m[zs[0]:zs[-1] + 1, ys[0]:ys[-1] + 1, xs[0]:xs[-1] + 1] |= ins.astype(np.uint8)
    return m


def link_wall_distances(grid, prims, mask=None, iters=40):
    """Wall distances of the links from fluid cells into obstacle cells (for
    the interpolated bounce-back): for each fluid cell x and direction c_j
    with x + c_j solid, q = |x_w - x| / |c_j| in (0, 1), x_w the crossing of
    the segment x -> x + c_j with the surface of the union of primitives
    (bisection of the inside test, `iters` halvings).  Directions are indexed
    i = (cx+1) + 3(cy+1) + 9(cz+1); cells are x + nx (y + ny z).

    Returns (cell, direction, q) arrays of the links (int64, int8, float64).
    Links leaving the grid are not obstacle links and are not listed."""
    nx, ny, nz = grid
    m = voxelize(grid, prims) if mask is None else mask
    solid = np.argwhere(m != 0)                      # [k, (z, y, x)]
    cells, dirs, qs = [], [], []
    for j in range(27):
        cx, cy, cz = j % 3 - 1, (j // 3) % 3 - 1, j // 9 - 1
        if cx == 0 and cy == 0 and cz == 0:
            continue
        # fluid cells x with x + c_j solid: x = s - c_j for solid s
        z, y, x = solid[:, 0] - cz, solid[:, 1] - cy, solid[:, 2] - cx
        ok = (x >= 0) & (x < nx) & (y >= 0) & (y < ny) & (z >= 0) & (z < nz)
        z, y, x = z[ok], y[ok], x[ok]
        ok = m[z, y, x] == 0
        z, y, x = z[ok], y[ok], x[ok]
        if len(x) == 0:
            continue
        lo = np.zeros(len(x))                        # outside at 0
        hi = np.ones(len(x))                         # inside at 1
        X0, Y0, Z0 = x.astype(np.float64), y.astype(np.float64), z.astype(np.float64)
        for _ in range(iters):
            mid = 0.5 * (lo + hi)
            X, Y, Z = X0 + mid * cx, Y0 + mid * cy, Z0 + mid * cz
            ins = np.zeros(len(x), bool)
            for pr in prims:
                ins |= pr.inside(X, Y, Z)
            hi = np.where(ins, mid, hi)
            lo = np.where(ins, lo, mid)
        cells.append(x + nx * (y + ny * z))
        dirs.append(np.full(len(x), j, np.int8))
        qs.append(0.5 * (lo + hi))
    if not cells:
        return np.zeros(0, np.int64), np.zeros(0, np.int8), np.zeros(0)
    return (np.concatenate(cells).astype(np.int64), np.concatenate(dirs), np.concatenate(qs))


def dense_wall_distances(grid, links):
    """[27, nz, ny, nx] array of q (1/2 where no obstacle link) from the
    (cell, direction, q) lists of link_wall_distances."""
    nx, ny, nz = grid
    q = np.full((27, nx * ny * nz), 0.5)
    cell, d, v = links
    q[d.astype(np.int64), cell] = v
    return q.reshape(27, nz, ny, nx)


def sphere(grid, center, radius) -> np.ndarray:
    return voxelize(grid, [Primitive("sphere", tuple(center), (2.0 * radius,))])


def cylinder_z(grid, center_xy, diameter) -> np.ndarray:
    """Spanwise cylinder: axis along z across the whole span."""
    nx, ny, nz = grid
    c = (center_xy[0], center_xy[1], 0.5 * (nz - 1))
    return voxelize(grid, [Primitive("cylinder", c, (float(diameter), float(nz + 2)))])


@dataclass
class Obstacle:
    grid: tuple
    prims: list = field(default_factory=list)
    angle_deg: float = 0.0
    seed: int = 0

    def mask(self) -> np.ndarray:
        return voxelize(self.grid, self.prims)


def composite(seed: int, grid, size_range=(20.0, 60.0), n_range=(2, 4),
              angle_range=(-30.0, 30.0), x_frac=0.3, jitter=10.0) -> Obstacle:
    """Union of 2-4 random primitives about (x_frac*nx, ny/2, nz/2), each
    size_range cells across, the whole composite turned by one angle of attack
    about z.  Deterministic in ``seed`` (NumPy PCG64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nx, ny, nz = grid
    n = int(rng.integers(n_range[0], n_range[1] + 1))
    alpha = float(rng.uniform(*angle_range))
    cx, cy, cz = x_frac * nx, 0.5 * (ny - 1), 0.5 * (nz - 1)
    lo, hi = size_range
    a = math.radians(alpha)
    prims = []
    for _ in range(n):
        kind = PRIMITIVES[int(rng.integers(0, len(PRIMITIVES)))]
        off = rng.uniform(-jitter, jitter, size=3)
        # the offset turns with the composite
        ox = math.cos(a) * off[0] - math.sin(a) * off[1]
        oy = math.sin(a) * off[0] + math.cos(a) * off[1]
        c = (cx + ox, cy + oy, cz + off[2])
        if kind == "sphere":
            size = (rng.uniform(lo, hi),)
        elif kind == "cylinder":
            size = (rng.uniform(lo, hi), rng.uniform(lo, hi))
        elif kind == "rectangle":
            size = tuple(rng.uniform(lo, hi, size=3))
        elif kind == "torus":
            d = rng.uniform(lo, hi)
            size = (d, rng.uniform(0.2, 0.4) * d)
        else:
            size = tuple(rng.uniform(lo, hi, size=3))
        prims.append(Primitive(kind, c, tuple(float(s) for s in size), alpha))
    return Obstacle(tuple(grid), prims, alpha, seed)


# ---------------------------------------------------------------------------
# workload recipes (inputs only: grids, obstacle, flow parameters)
# ---------------------------------------------------------------------------
def sphere_channel_64():
    """64x32x32 channel, sphere of radius 4 cells at x=16 centred in y, z;
    inlet u = 0.05, Re = 1000 on the sphere diameter."""
    grid = (64, 32, 32)
    return dict(grid=grid, mask=sphere(grid, (16.0, 15.5, 15.5), 4.0),
                re=1000.0, u_in=0.05, l_ref=8.0)


def cylinder_channel_256():
    """256x128x128 channel, spanwise cylinder of diameter 16 at x=64, Re=3900
    on the diameter, u = 0.05."""
    grid = (256, 128, 128)
    return dict(grid=grid, mask=cylinder_z(grid, (64.0, 63.5), 16.0),
                re=3900.0, u_in=0.05, l_ref=16.0)


def composite_channel(seed=0, grid=(1024, 512, 512), re=10000.0, u_in=0.05):
    """Full-size channel with a seeded composite obstacle; Re on the channel
    height."""
    obs = composite(seed, grid)
    return dict(grid=tuple(grid), mask=obs.mask(), re=re, u_in=u_in,
                l_ref=float(grid[1]), angle_deg=obs.angle_deg, obstacle=obs)


def batch_channels(seed=0, n=32, u_in=0.05):
    """Uneven grids from {128,192,256} x {64,96,128}^2, Re log-uniform in
    [1000, 10000] on the channel height, composite obstacles scaled by
    ny/512 (floor 6 cells)."""
    rng = np.random.Generator(np.random.PCG64(10_000 + seed))
    out = []
    for g in range(n):
        grid = (int(rng.choice([128, 192, 256])), int(rng.choice([64, 96, 128])),
                int(rng.choice([64, 96, 128])))
        re = float(math.exp(rng.uniform(math.log(1000.0), math.log(10000.0))))
        s = grid[1] / 512.0
        lo, hi = max(6.0, 20.0 * s), max(6.0, 60.0 * s)
        obs = composite(seed * 1000 + g, grid, size_range=(lo, hi), jitter=10.0 * s)
        out.append(dict(grid=grid, mask=obs.mask(), re=re, u_in=u_in,
                        l_ref=float(grid[1]), angle_deg=obs.angle_deg, obstacle=obs))
    return out
