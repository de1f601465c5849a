"""Batched driver: graph-captured batched launches over uneven grids must give
exactly what independent contexts give (same kernels per cell, same
arithmetic order, deterministic force reductions), members must stop at their
own end, and the autotuners must leave the lattices at rest."""
import numpy as np
import pytest

import oracle.lbm as O
from paper_2606_16765_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_16765_gb300 import _build
    _build.build()


def members(storage="f32", mean=True, force=True):
    out = []
    for g, (grid, w1) in enumerate([((40, 16, 12), 1.6), ((64, 20, 16), 1.85), ((96, 12, 12), 1.95),
                                    ((33, 9, 7), 1.3)]):
        nx, ny, nz = grid
        mask = I.sphere(grid, (0.3 * nx, 0.5 * (ny - 1), 0.5 * (nz - 1)), 0.22 * ny)
        d = dict(grid=grid, mask=mask, storage=storage, omega1=w1, u_in=0.05)
        if mean:
            d.update(mean_start=4, mean_end=1000, mean_every=2)
        if force:
            d.update(force_every=1, force_capacity=4096)
        out.append(d)
    return out


def independent(d, steps, **extra):
    """The member's lattice stepped alone, with the member's own options (the
    same cell classes, hence the same force-reduction blocks and bits)."""
    from paper_2606_16765_gb300.lbm import Solver
    kw = {k: v for k, v in d.items() if k not in ("grid", "mask")}
    kw.update(extra)
    s = Solver(d["grid"], d["mask"], **kw)
    s.step(steps)
    s.sync()
    return s


@pytest.mark.parametrize("storage", ["f32", "f16s"])
def test_batch_equals_independent_runs(storage):
    from paper_2606_16765_gb300.lbm import Batch
    ms = members(storage)
    b = Batch(ms)
    b.run(20)
    b.sync()
    info = b.info()
    assert info.t == 20 and info.graph_captures == 1 and info.graph_launches == 10
    for g, d in enumerate(ms):
        m = b.member(g)
        ref = independent(d, 20)
        assert m.t == 20
        assert np.array_equal(m.pdfs(), ref.pdfs()), g
        ma, sa = m.mean()
        mb, sb = ref.mean()
        assert sa == sb == 8 and np.array_equal(ma, mb)
        assert np.array_equal(m.forces(), ref.forces())


def test_members_stop_at_their_end():
    from paper_2606_16765_gb300.lbm import Batch
    ms = members("f32", mean=False, force=False)
    b = Batch(ms)
    ends = [6, 14, 20, 2]
    b.set_end(ends)
    b.run_to_end()
    b.sync()
    info = b.info()
    assert info.live == 0 and info.t == 20
    assert info.graph_captures == 4          # live sets {0,1,2,3}, {0,1,2}, {1,2}, {2}
    for g, d in enumerate(ms):
        m = b.member(g)
        assert m.t == ends[g]
        assert np.array_equal(m.pdfs(), independent(d, ends[g]).pdfs()), g


def test_flowthrough_ends():
    from paper_2606_16765_gb300.lbm import Batch
    ms = members("f32", mean=False, force=False)
    b = Batch(ms)
    b.set_flowthroughs(0.05)                  # 0.05 * nx / 0.05 = nx steps, rounded to the chunk
    b.run_to_end()
    b.sync()
    for g, d in enumerate(ms):
        nx = d["grid"][0]
        assert b.member(g).t == nx + (nx % 2)


def test_batch_autotune_resets_to_rest_and_runs_with_the_choice():
    from paper_2606_16765_gb300.lbm import Batch
    ms = members("f32")
    b = Batch(ms)
    bx, by, ms_step = b.autotune(trials=2)
    assert bx % 32 == 0 and bx * by <= 256 and ms_step > 0
    info = b.info()
    assert info.t == 0 and info.block_x == bx and info.block_y == by
    w = O.weights()
    for g in range(len(ms)):
        f = b.member(g).pdfs()
        assert np.abs(f - w[:, None, None, None]).max() == 0.0
    b.run(10)
    b.sync()
    for g, d in enumerate(ms):
        ref = independent(d, 10, block_x=bx, block_y=by)
        assert np.array_equal(b.member(g).pdfs(), ref.pdfs())


def test_single_context_autotune():
    from paper_2606_16765_gb300.lbm import Solver
    d = members("f32")[1]
    s = Solver(d["grid"], d["mask"], storage="f32", omega1=1.8, u_in=0.05, mean_start=0, mean_end=100,
               mean_every=2, force_every=1)
    bx, by, t = s.autotune(trials=4)
    assert bx % 32 == 0 and bx * by <= 256 and t > 0
    assert s.t == 0 and s.forces().shape == (0, 3)
    w = O.weights()
    assert np.abs(s.pdfs() - w[:, None, None, None]).max() == 0.0


def test_batch_argument_errors():
    from paper_2606_16765_gb300.lbm import Batch, LBMError
    ms = members("f32")
    ms[1]["storage"] = "f16s"
    with pytest.raises(LBMError):
        Batch(ms)
    ms = members("f32")
    ms[2]["mean_every"] = 4
    with pytest.raises(LBMError):
        Batch(ms)
    ms = members("f32")
    ms[0]["snap_count"] = 2
    ms[0]["snap_every"] = 5
    with pytest.raises(LBMError):
        Batch(ms)


def test_lowest_viscosity_members_reach_fifteen_flowthroughs():
    """The eight members of the 32-channel batch with the smallest lattice
    viscosity (nu = 3.3e-4 .. 8.7e-4, omega1 up to 1.996) run together to 15
    flow-through times in FP16S storage with the convective outflow; none
    latches an instability and every time average is finite."""
    from paper_2606_16765_gb300.lbm import Batch
    chans = I.batch_channels(0, n=32)
    nu = [d["u_in"] * d["l_ref"] / d["re"] for d in chans]
    pick = sorted(range(len(chans)), key=lambda g: nu[g])[:8]
    ms = []
    for g in pick:
        d = chans[g]
        t_end = int(np.ceil(15 * d["grid"][0] / d["u_in"]))
        ms.append(dict(grid=d["grid"], mask=d["mask"], storage="f16s", re=d["re"], u_in=d["u_in"], l_ref=d["l_ref"],
                       mean_start=int(round(5 * d["grid"][0] / d["u_in"] / 10)) * 10, mean_end=t_end, mean_every=10))
    b = Batch(ms)
    b.set_flowthroughs(15.0)
    b.run_to_end()
    b.sync()
    info = b.info()
    assert info.live == 0
    for k, g in enumerate(pick):
        m, ns = b.member(k).mean(halfres=True, dtype=np.float32)
        assert ns > 0 and np.isfinite(m).all(), g
        fl = m[..., 0][np.isfinite(m[..., 0])]
        assert 0.0 < float(np.median(fl)) < 0.1, g
    b.close()


def test_batch_with_wall_distances_equals_independent_runs():
    """Interpolated bounce-back in a batch (end-of-step kernel, one block per
    member) against the same lattices stepped alone (their own kernel):
    populations bitwise equal; the force corrections are reduced in another
    order, so the force rows agree to rounding."""
    from paper_2606_16765_gb300.lbm import Batch, Solver
    ms = members("f32")
    links = []
    for d in ms:
        nx, ny, nz = d["grid"]
        prim = I.Primitive("sphere", (0.3 * nx, 0.5 * (ny - 1), 0.5 * (nz - 1)), (0.44 * ny,))
        links.append(I.link_wall_distances(d["grid"], [prim], d["mask"]))
    b = Batch(ms)
    for g in range(len(ms)):
        b.set_wall_distances(g, links[g])
    b.run(20)
    b.sync()
    for g, d in enumerate(ms):
        kw = {k: v for k, v in d.items() if k not in ("grid", "mask")}
        s = Solver(d["grid"], d["mask"], **kw)
        s.set_wall_distances(links[g])
        s.step(20)
        s.sync()
        m = b.member(g)
        assert np.array_equal(m.pdfs(), s.pdfs()), g
        Fa, Fb = m.forces(), s.forces()
        assert Fa.shape == Fb.shape
        assert np.abs(Fa - Fb).max() <= 1e-12 * np.abs(Fb).max(), g


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_batch_members_match_the_oracle(storage):
    """Three members on uneven small grids stepped by the batched driver, each
    compared directly with the FP64 oracle run of its own lattice: convective
    outflow, interpolated bounce-back on the obstacle links (wall distances
    of the primitives), FP64 mean and force records.  FP64 pdfs to 1e-12,
    FP32 to 1e-5 (max relative velocity error and density error)."""
    from paper_2606_16765_gb300.lbm import Batch
    faces = ("inlet", "outflow", "wall", "wall")
    specs = [((40, 16, 12), 1.6, I.Primitive("sphere", (12.0, 7.5, 5.5), (7.0,))),
             ((57, 21, 14), 1.85, I.Primitive("cylinder", (17.3, 10.2, 6.5), (6.4, 9.0), 12.0)),
             ((26, 9, 11), 1.3, I.Primitive("torus", (8.0, 4.1, 5.0), (6.5, 2.2)))]
    steps = 30
    ms, refs = [], []
    for grid, w1, prim in specs:
        nx, ny, nz = grid
        mask = I.voxelize(grid, [prim])
        links = I.link_wall_distances(grid, [prim], mask)
        ms.append(dict(grid=grid, mask=mask, storage=storage, omega1=w1, u_in=0.05, faces=faces,
                       mean_start=10, mean_end=1000, mean_every=2, force_every=1, force_capacity=256))
        L = O.Lattice(O.params(nx, ny, nz, w1, u_in=0.05, faces=faces, mean=(10, 1000, 2)), mask)
        L.set_q(I.dense_wall_distances(grid, links))
        L.step(steps)
        refs.append((L, mask, links))
    b = Batch(ms)
    for g, (_, _, links) in enumerate(refs):
        b.set_wall_distances(g, links)
    b.run(steps)
    b.sync()
    tol = {"f64": 1e-12, "f32": 1e-5}[storage]
    for g, (L, mask, links) in enumerate(refs):
        m = b.member(g)
        assert m.t == steps
        fl = mask == 0
        rho, u = m.macros()
        rr, ur = L.macros()
        eu = np.abs(u - ur)[fl].max() / np.abs(ur[fl]).max()
        er = np.abs(rho - rr)[fl].max()
        mean, ns = m.mean()
        mref, nref = L.means()
        em = np.abs(mean - mref)[fl].max() / np.abs(mref[..., :3])[fl].max()
        F, Fr = m.forces(), L.forces()
        ef = np.abs(F - Fr).max() / np.abs(Fr).max()
        print(f"batch member {g} {storage}: u {eu:.2e} rho {er:.2e} mean {em:.2e} force {ef:.2e}, "
              f"{len(links[0])} wall-distance links")
        assert eu <= tol and er <= tol and em <= tol
        assert ns == nref == 10
        assert F.shape == Fr.shape == (steps, 3) and ef <= 10 * tol
