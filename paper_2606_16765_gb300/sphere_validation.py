"""Sphere-in-channel validation runs of the solver (Sec. 3.3, Table 1).

The paper validates its solver on a sphere in the same 2 x 1 x 1 channel as
the dataset: diameter D = L/6 of the channel height L (so Re_c = 6 Re_s), at
x = 0.6 L (x/2L = 0.3), centred in y and z, uniform inlet velocity,
extrapolating outflow, no-slip walls.  Table 1 gives the drag coefficient
C_d = F_x / (rho U^2 pi D^2 / 8) at resolutions L = 128 ... 1024 cells; at
Re_s = 1000 the paper also reports the recirculation length (l_r/D = 1.8),
the Strouhal number of the vertical wake velocity (St ~ 0.18) and the two
peaks of u'_rms on the centreline (x/D = 1.5 and 2.4 behind the centre).

  python -m paper_2606_16765_gb300.sphere_validation [--cases 128:100,128:500] [--wake 256] [--out f.json]

Every run starts from rest with the solver's default boundary set
(moving-wall inlet, convective outflow, walls) and the interpolated
bounce-back on the sphere's links (wall distances from the exact sphere).
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import inputs as I
from . import wake

U = 0.05

# Table 1: drag coefficient at resolution L (cells per channel height)
TABLE1 = {
    100: {128: 1.122, 256: 1.108, 384: 1.106, 512: 1.106},
    500: {128: 0.573, 256: 0.562, 384: 0.563, 512: 0.562},
    1000: {128: 0.479, 256: 0.460, 384: 0.466, 512: 0.467, 1024: 0.472},
    2000: {128: 0.434, 256: 0.407, 384: 0.407, 512: 0.404},
}


def sphere_channel(L):
    """Grid, diameter, centre, primitives, mask and wall-distance links of
    the validation channel at resolution L."""
    grid = (2 * L, L, L)
    D = L / 6.0
    c = (0.6 * L, 0.5 * (L - 1), 0.5 * (L - 1))
    prims = [I.Primitive("sphere", c, (D,))]
    mask = I.voxelize(grid, prims)
    return grid, D, c, prims, mask, I.link_wall_distances(grid, prims, mask)


def centreline(field, c):
    """Profile along x of a [nz, ny, nx] field on the axis through c = (x, y, z)
    (cell centres): the mean of the four rows around (c[1], c[2])."""
    y0, y1 = int(math.floor(c[1])), int(math.ceil(c[1]))
    z0, z1 = int(math.floor(c[2])), int(math.ceil(c[2]))
    return 0.25 * (field[z0, y0] + field[z0, y1] + field[z1, y0] + field[z1, y1])


def profile_peaks(values, xs, lo, hi, count=2):
    """Positions xs of the `count` largest local maxima of a profile with
    lo < xs < hi, in increasing order of position."""
    idx = np.nonzero((xs > lo) & (xs < hi))[0]
    v = values[idx]
    peaks = [i for i in range(1, len(v) - 1) if v[i] >= v[i - 1] and v[i] >= v[i + 1]]
    top = sorted(peaks, key=lambda i: -v[i])[:count]
    return sorted(float(xs[idx[i]]) for i in top)


def drag_coefficient(fx, D):
    """C_d of the sphere from a streamwise force record."""
    return float(np.mean(fx)) / (0.5 * U * U * math.pi * D * D / 4.0)


def drag_run(L, re, n_ft=10.0, avg_from_ft=5.0, storage="f32", every=10, lateral="wall"):
    """C_d at resolution L and Re_s: the mean force over flow-through times
    [avg_from_ft, n_ft) of a run from rest; also the C_d of each flow-through
    window, to judge convergence.  lateral = "wall" (no-slip channel walls,
    the paper's set-up) or "periodic" (y and z wrap around: a sphere in a
    periodic array of spacing 6 D, free of wall boundary layers)."""
    from .lbm import Solver

    grid, D, _, _, mask, links = sphere_channel(L)
    ft = 2 * L / U
    steps = int(round(n_ft * ft / every)) * every
    s = Solver(grid, mask, storage=storage, re=float(re), u_in=U, l_ref=D, force_every=every,
               force_capacity=steps // every + 1, faces=("inlet", "outflow", lateral, lateral))
    try:
        s.set_wall_distances(links)
        t0 = time.time()
        s.step(steps)
        s.sync()
        sec = time.time() - t0
        F = s.forces()
    finally:
        s.close()
    rows_per_ft = ft / every
    k0 = int(round(avg_from_ft * rows_per_ft))
    windows = [drag_coefficient(F[int(k * rows_per_ft):int((k + 1) * rows_per_ft), 0], D)
               for k in range(int(n_ft))]
    return dict(L=L, re_s=re, lateral=lateral, cd=drag_coefficient(F[k0:, 0], D), cd_per_ft=windows,
                steps=steps, seconds=sec, links=int(len(links[0])))


def wake_run(L, re=1000.0, n_ft=12.0, mean_from_ft=4.0, storage="f32", probe_every=10, mean_every=10):
    """Re_s = 1000 wake measures at resolution L: C_d, St of the vertical
    velocity at probes behind the sphere, l_r/D of the mean centreline
    velocity and the positions of the u'_rms peaks on the centreline."""
    from .lbm import Solver

    grid, D, c, _, mask, links = sphere_channel(L)
    nx, ny, nz = grid
    ft = 2 * L / U
    steps = int(round(n_ft * ft / mean_every)) * mean_every
    t0s = int(round(mean_from_ft * ft / mean_every)) * mean_every
    s = Solver(grid, mask, storage=storage, re=float(re), u_in=U, l_ref=D, force_every=probe_every,
               force_capacity=steps // probe_every + 1, mean_start=t0s, mean_end=steps, mean_every=mean_every,
               stats=1)
    try:
        s.set_wall_distances(links)
        # probes in the mid-span plane, half a diameter off the axis, 1-3 D behind the centre
        jy, kz = int(round(c[1] + 0.5 * D)), int(round(c[2]))
        px = [int(round(c[0] + a * D)) for a in (1.0, 1.5, 2.0, 3.0)]
        cells = np.array([x + nx * (jy + ny * kz) for x in px], np.int64)
        s.set_probes(cells, every=probe_every, capacity=steps // probe_every + 1)
        t0 = time.time()
        s.step(steps)
        s.sync()
        sec = time.time() - t0
        F = s.forces()
        P = s.probes()
        m, ns = s.mean(dtype=np.float32)
        st, _ = s.stats(dtype=np.float32)
    finally:
        s.close()
    k0 = t0s // probe_every
    cd = drag_coefficient(F[k0:, 0], D)
    sts = [float(wake.strouhal(P[k0:, j, 1], D, U, every=probe_every, st_band=(0.05, 0.5))) for j in range(len(px))]
    u_c = centreline(m[..., 0], c)
    lr = wake.recirculation_length(u_c, c[0] + 0.5 * D) / D
    urms = np.sqrt(np.maximum(centreline(st[..., 0], c), 0.0)) / U
    xs = (np.arange(nx) - c[0]) / D
    behind = (xs > 0.5) & (xs < 5.0)
    return dict(L=L, re_s=re, cd=cd, st_probes=sts, probe_x_over_d=[(x - c[0]) / D for x in px], lr_over_d=lr,
                urms_peaks_x_over_d=profile_peaks(urms, xs, 0.5, 5.0), urms_max=float(urms[behind].max()),
                mean_samples=int(ns), steps=steps,
                seconds=sec, centreline_u=[float(v) for v in u_c / U],
                centreline_urms=[float(v) for v in urms])


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--cases", default="128:100,128:500,128:1000,128:2000,256:100,256:500",
                    help="comma list of L:Re_s drag runs")
    ap.add_argument("--wake", type=int, default=0, help="resolution L of the Re_s = 1000 wake run (0: none)")
    ap.add_argument("--n-ft", type=float, default=10.0)
    ap.add_argument("--lateral", default="wall", choices=["wall", "periodic"],
                    help="y/z faces of the drag runs (the wake run always has walls)")
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    rep = {"drag": [], "wake": None}
    for cs in filter(None, a.cases.split(",")):
        L, re = (int(v) for v in cs.split(":"))
        r = drag_run(L, re, n_ft=a.n_ft, lateral=a.lateral)
        r["paper"] = TABLE1.get(re, {}).get(L)
        rep["drag"].append(r)
        print(f"L {L} Re_s {re} ({a.lateral}): C_d {r['cd']:.4f} (paper {r['paper']}), per flow-through "
              f"{[round(v, 4) for v in r['cd_per_ft']]}, {r['seconds']:.1f} s", flush=True)
        if a.out:
            with open(a.out, "w") as fp:
                json.dump(rep, fp, indent=1)
    if a.wake:
        w = wake_run(a.wake)
        rep["wake"] = w
        print(f"wake L {a.wake} Re_s 1000: C_d {w['cd']:.4f}, St {[round(v, 3) for v in w['st_probes']]}, "
              f"l_r/D {w['lr_over_d']:.3f}, u'_rms peaks at x/D {w['urms_peaks_x_over_d']}, {w['seconds']:.1f} s",
              flush=True)
    if a.out:
        with open(a.out, "w") as fp:
            json.dump(rep, fp, indent=1)
    return rep


if __name__ == "__main__":
    main()
