"""GPU parity of the CUDA D3Q27 cumulant step against the FP64 oracle.

Every case runs the same seeded inputs through the C ABI (via the thin
binding) and through the oracle, and compares element by element:
  FP64 pdfs   <= 1e-12 (max relative velocity error, density error),
  FP32 pdfs   <= 1e-5  (sphere channel, 200 steps from rest),
  F16C pdfs   <= 1e-3 (the FP16-shifted format that meets the 1e-3 bound:
                       a 16-bit float with 4 exponent and 11 mantissa bits),
on the 64x32x32 sphere channel; IEEE binary16 (FP16S, one mantissa bit less)
and bfloat16 (BF16S) are secondary formats whose errors are reported, not
held to that bound; small boxes cover every boundary kind, the
general (omega_higher != 1) and uncorrected collision variants, ragged grids
and degenerate sizes; the 1024x512x512 channel is checked on sampled cells.
"""
import os

import numpy as np
import pytest

import oracle.lbm as O
from paper_2606_16765_gb300 import inputs as I
from tests import cases as K

pytestmark = pytest.mark.gpu

# FP16-shifted storage is held to 1e-3 through F16C, whose 12 significant
# bits halve the storage rounding of IEEE binary16 (11 bits); binary16 itself
# measures 0.7-1.2e-3 on the sphere channel, above that bound, and is reported.
TOL_U = {"f64": 1e-12, "f32": 1e-5, "f16c": 1e-3}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_16765_gb300 import _build
    _build.build()


# --------------------------------------------------------------------------
# sphere channel 64x32x32, 200 steps from rest (Re = 1000 on the diameter)
# --------------------------------------------------------------------------
@pytest.fixture(scope="module")
def sphere64():
    d = I.sphere_channel_64()
    w1 = O.omega_from_re(d["re"], d["u_in"], d["l_ref"])
    c = K.case(d["grid"], d["mask"], omega1=w1, u_in=d["u_in"], mean=(100, 200, 1))
    L = K.run_oracle(c, 200)
    rho, u = L.macros()
    f = L.get_f()
    means, s = L.means()
    return dict(case=c, rho=rho, u=u, f=f, means=means, samples=s, forces=L.forces())


@pytest.mark.parametrize("storage", ["f64", "f32", "f16c"])
def test_sphere_channel_200_steps(sphere64, storage):
    c = sphere64["case"]
    s = K.make_solver(c, storage, force_every=1)
    s.step(200)
    s.sync()
    rho, u = s.macros()
    fluid = c["mask"] == 0
    eu = K.rel_u_err(u, sphere64["u"], fluid)
    er = K.rho_err(rho, sphere64["rho"], fluid)
    print(f"{storage}: rel u err {eu:.3e}  rho err {er:.3e}")
    assert eu <= TOL_U[storage]
    assert er <= TOL_U[storage]
    if storage == "f64":
        f = s.pdfs()
        assert np.abs(f - sphere64["f"])[:, fluid].max() < 1e-13
    # time average over steps 100..199 and the force series
    m, ns = s.mean()
    assert ns == sphere64["samples"] == 100
    mref = sphere64["means"]
    em = np.abs(m - mref)[fluid].max() / np.abs(mref[..., :3])[fluid].max()
    assert em <= TOL_U[storage]
    F = s.forces()
    Fr = sphere64["forces"]
    assert F.shape == Fr.shape == (200, 3)
    assert np.abs(F - Fr).max() <= TOL_U[storage] * np.abs(Fr[:, 0]).max() * 10


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_sphere_channel_outflow_200_steps(storage):
    """The same channel with the convective outflow on the x-high face."""
    d = I.sphere_channel_64()
    w1 = O.omega_from_re(d["re"], d["u_in"], d["l_ref"])
    c = K.case(d["grid"], d["mask"], omega1=w1, u_in=d["u_in"], faces=("inlet", "outflow", "wall", "wall"))
    L = K.run_oracle(c, 200)
    rho_r, u_r = L.macros()
    s = K.make_solver(c, storage)
    s.step(200)
    s.sync()
    rho, u = s.macros()
    fluid = c["mask"] == 0
    eu, er = K.rel_u_err(u, u_r, fluid), K.rho_err(rho, rho_r, fluid)
    print(f"outflow {storage}: rel u err {eu:.3e}  rho err {er:.3e}")
    assert eu <= TOL_U[storage] and er <= TOL_U[storage]


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_velocity_statistics_match_oracle(storage):
    """Reynolds-stress accumulators (FP64 sums of velocity products over the
    averaging samples) against the oracle's, over the start-up of the sphere
    channel from a noisy state (large fluctuations)."""
    d = I.sphere_channel_64()
    w1 = O.omega_from_re(d["re"], d["u_in"], d["l_ref"])
    c = K.case(d["grid"], d["mask"], omega1=w1, u_in=d["u_in"], faces=("inlet", "outflow", "wall", "wall"),
               mean=(20, 120, 2), noise=(31, 2e-3))
    L = K.run_oracle(c, 120)
    ref, n = L.stats()
    s = K.make_solver(c, storage, stats=1)
    s.step(120)
    s.sync()
    st, ns = s.stats()
    assert ns == n == 50
    fl = c["mask"] == 0
    err = np.abs(st - ref)[fl].max() / np.abs(ref[fl]).max()
    print(f"stats {storage}: max rel err {err:.3e}, max covariance {np.abs(ref[fl]).max():.3e}")
    assert err <= {"f64": 1e-8, "f32": 1e-4}[storage]


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_probes_record_the_state_before_each_sampled_step(storage):
    """Probe rows against the oracle's macros of the state before the step,
    every third step for 40 steps, at wake, inlet, outlet and solid cells."""
    d = I.sphere_channel_64()
    nx, ny, nz = d["grid"]
    w1 = O.omega_from_re(d["re"], d["u_in"], d["l_ref"])
    c = K.case(d["grid"], d["mask"], omega1=w1, u_in=d["u_in"], faces=("inlet", "outflow", "wall", "wall"),
               noise=(33, 1e-3))
    pts = [(24, 15, 16), (0, 3, 30), (nx - 1, 16, 16), (nx - 1, 0, 0), (16, 15, 15), (40, 31, 0)]
    cells = np.array([x + nx * (y + ny * z) for x, y, z in pts], np.int64)
    s = K.make_solver(c, storage)
    s.set_probes(cells, every=3, capacity=4)          # several flushes to the host
    s.step(40)
    s.sync()
    rec = s.probes()
    assert rec.shape == (14, len(cells), 4)
    L = K.run_oracle(c, 0)
    ref = []
    for t in range(40):
        if t % 3 == 0:
            rho, u = L.macros()
            z, y, x = np.unravel_index(cells, (nz, ny, nx))
            row = np.concatenate([u[z, y, x], ((rho[z, y, x] - 1) / 3)[:, None]], 1)
            row[d["mask"][z, y, x] != 0] = 0.0
            ref.append(row)
        L.step(1)
    ref = np.array(ref)
    err = np.abs(rec - ref).max() / np.abs(ref[..., :3]).max()
    print(f"probes {storage}: max rel err {err:.2e}")
    assert err <= (2e-6 if storage == "f64" else 1e-5)
    assert np.all(rec[:, 4] == 0)                     # the solid cell


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_equilibrium_initialisation_matches_oracle_equilibrium(storage):
    """lbm_init_equilibrium against the oracle's product-form equilibrium at
    rho = 1 + 3 p and u, cell by cell (solid cells at rest)."""
    from paper_2606_16765_gb300.lbm import Solver
    g = (13, 7, 5)
    mask = I.sphere(g, (6.0, 3.0, 2.0), 1.6)
    r = np.random.default_rng(4)
    fields = np.concatenate([r.uniform(-0.08, 0.08, (5, 7, 13, 3)), r.uniform(-0.01, 0.01, (5, 7, 13, 1))], -1)
    fields = fields.astype(np.float32)
    s = Solver(g, mask, storage=storage, omega1=1.5)
    s.init_equilibrium(fields)
    f = s.pdfs()
    w = O.weights()
    err = 0.0
    for z, y, x in np.ndindex(5, 7, 13):
        if mask[z, y, x]:
            ref = w
        else:
            u = fields[z, y, x].astype(np.float64)
            ref = np.asarray(O.equilibrium(1.0 + 3.0 * u[3], u[0], u[1], u[2]))
        err = max(err, np.abs(f[:, z, y, x] - ref).max())
    assert err <= (1e-15 if storage == "f64" else 1e-8)


def test_outflow_keeps_low_viscosity_channel_stable():
    """An empty 128x64x128 channel at nu = 3.3e-4 (the thinnest member of the
    32-channel batch): with the anti-bounce-back outlet it diverges within
    400 steps; with the convective outflow it runs 4000 steps."""
    from paper_2606_16765_gb300.lbm import LBMError, Solver
    nu = 3.3e-4
    s = Solver((128, 64, 128), None, storage="f32", omega1=1.0 / (3 * nu + 0.5), u_in=0.05)
    s.step(4000)
    s.sync()
    rho, u = s.macros()
    assert np.isfinite(rho).all() and np.abs(rho - 1).max() < 0.2
    a = Solver((128, 64, 128), None, storage="f32", omega1=1.0 / (3 * nu + 0.5), u_in=0.05,
               faces=("inlet", "outlet", "wall", "wall"))
    a.step(1000)
    with pytest.raises(LBMError):
        a.sync()


@pytest.mark.parametrize("storage", ["f16s", "bf16s"])
def test_secondary_16bit_formats_run_and_are_reported(sphere64, storage):
    """IEEE binary16 (11 significant bits) and bfloat16 (8) shifted storage:
    their error against the oracle is reported, not gated at 1e-3 (binary16
    measures about 1e-3, bfloat16 about 1e-2).  The assertion only catches a
    broken path: finite and within 10x the bound's scale of each format."""
    c = sphere64["case"]
    s = K.make_solver(c, storage)
    s.step(200)
    s.sync()
    rho, u = s.macros()
    fluid = c["mask"] == 0
    eu = K.rel_u_err(u, sphere64["u"], fluid)
    er = K.rho_err(rho, sphere64["rho"], fluid)
    print(f"{storage}: rel u err {eu:.3e}  rho err {er:.3e}  (reported; 1e-3 is met by f16c)")
    assert np.isfinite(eu) and eu < {"f16s": 1e-2, "bf16s": 0.5}[storage]


# --------------------------------------------------------------------------
# small boxes: every boundary kind, ragged sizes, both collision variants
# --------------------------------------------------------------------------
def box_cases():
    g = (37, 13, 11)                     # ragged: not a multiple of the block
    obs = I.sphere(g, (9.0, 6.0, 5.0), 3.0)
    wall_obs = I.voxelize(g, [I.Primitive("rectangle", (20.0, 1.0, 5.0), (4.0, 4.0, 20.0))])  # touches y=0 and both z walls
    # solid cells in the outlet plane and next to it (the outflow's inner neighbour)
    outlet_obs = I.voxelize(g, [I.Primitive("rectangle", (35.5, 6.0, 5.0), (2.0, 4.0, 4.0))])
    return {
        "channel_obstacle": K.case(g, obs, omega1=1.7, noise=(11, 2e-3)),
        "obstacle_on_walls": K.case(g, wall_obs, omega1=1.9, noise=(12, 2e-3)),
        "periodic_all": K.case((9, 7, 5), None, omega1=1.3, faces=("periodic",) * 4, u_in=0.0, noise=(13, 5e-3)),
        "periodic_yz_inlet": K.case(g, obs, omega1=1.6, faces=("inlet", "outlet", "periodic", "periodic"), noise=(14, 2e-3)),
        "closed_box": K.case((12, 10, 8), I.sphere((12, 10, 8), (5.5, 4.5, 3.5), 2.0), omega1=1.95,
                             faces=("wall", "wall", "wall", "wall"), u_in=0.0, noise=(15, 3e-3)),
        "general_omega_higher": K.case(g, obs, omega1=1.5, omega_bulk=1.2, omega_higher=1.3, noise=(16, 2e-3)),
        "no_galilean": K.case(g, obs, omega1=1.8, galilean=0, noise=(17, 2e-3)),
        "thin_slab": K.case((16, 1, 3), None, omega1=1.4, faces=("inlet", "outlet", "periodic", "wall"), noise=(18, 2e-3)),
        "single_cell": K.case((1, 1, 1), None, omega1=1.1, faces=("periodic",) * 4, u_in=0.0, noise=(19, 5e-3)),
        # convective outflow on the x-high face
        "outflow_obstacle": K.case(g, obs, omega1=1.9, faces=OUTFLOW, noise=(20, 2e-3)),
        "outflow_solid_at_outlet": K.case(g, outlet_obs, omega1=1.8, faces=OUTFLOW, noise=(21, 2e-3)),
        "outflow_periodic_yz": K.case(g, obs, omega1=1.7, faces=("inlet", "outflow", "periodic", "periodic"),
                                      noise=(22, 2e-3)),
        "outflow_nx2": K.case((2, 5, 4), None, omega1=1.5, faces=OUTFLOW, noise=(23, 2e-3)),
        "outflow_nx1": K.case((1, 3, 3), None, omega1=1.5, faces=OUTFLOW, noise=(24, 2e-3)),
        # wall-row kernel: rows y = 0 and y = ny - 1 adjacent (ny = nz = 2),
        # one periodic lateral face, rows longer than one block (nx > 128)
        "wall_rows_2x2": K.case((20, 2, 2), None, omega1=1.6, faces=OUTFLOW, noise=(25, 2e-3)),
        "wall_y_periodic_z": K.case(g, obs, omega1=1.7, faces=("inlet", "outflow", "wall", "periodic"),
                                    noise=(26, 2e-3)),
        "wall_rows_long": K.case((150, 6, 4), I.sphere((150, 6, 4), (40.0, 2.5, 1.5), 1.5), omega1=1.8,
                                 faces=OUTFLOW, noise=(27, 2e-3)),
    }


OUTFLOW = ("inlet", "outflow", "wall", "wall")
BOXES = box_cases()


@pytest.mark.parametrize("name", sorted(BOXES))
@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_small_boxes(name, storage):
    c = BOXES[name]
    fluid = np.ones(c["grid"][::-1], bool) if c["mask"] is None else c["mask"] == 0
    s = K.make_solver(c, storage)
    L = K.run_oracle(c, 0)
    for steps in (1, 1, 5, 13):          # odd and even counts: both AA parities
        s.step(steps)
        L.step(steps)
        f = s.pdfs()
        fr = L.get_f()
        err = np.abs(f - fr)[:, fluid].max()
        tol = 1e-14 if storage == "f64" else 2e-7
        assert err <= tol, (name, storage, L.t, err)
    s.sync()


def test_cell_classes_cover_the_fluid():
    # every fluid cell is updated by exactly one of the bulk, wall-row and
    # edge kernels; a walled channel has wall-row cells, a periodic one none
    g = (37, 13, 11)
    obs = I.sphere(g, (9.0, 6.0, 5.0), 3.0)
    s = K.make_solver(K.case(g, obs, faces=OUTFLOW), "f32")
    i = s.info()
    assert i.fluid_cells == int((obs == 0).sum())
    assert i.bulk_cells + i.wall_cells + i.edge_cells == i.fluid_cells
    # rows next to the four walls, minus the x-face corners and the cells next to the sphere
    assert 0 < i.wall_cells <= 2 * (g[0] - 2) * (g[1] + g[2] - 2)
    p = K.make_solver(K.case(g, obs, faces=("inlet", "outflow", "periodic", "periodic")), "f32").info()
    assert p.wall_cells == 0 and p.bulk_cells + p.edge_cells == p.fluid_cells


def test_plain_fast_path_equals_general_path():
    """omega_higher = 1 takes the raw-moment fast path; an omega_higher one
    rounding step away takes the general cumulant path.  Both must agree."""
    d = I.sphere_channel_64()
    a = K.make_solver(K.case(d["grid"], d["mask"], omega1=1.95, noise=(9, 2e-3)), "f64")
    b = K.make_solver(K.case(d["grid"], d["mask"], omega1=1.95, omega_higher=1.0 + 2.0 ** -50,
                             noise=(9, 2e-3)), "f64")
    a.step(31)
    b.step(31)
    fl = d["mask"] == 0
    assert np.abs(a.pdfs() - b.pdfs())[:, fl].max() < 1e-13


def f16c_round(x32):
    """Nearest value of the 16-bit custom float (4 exponent bits, bias 15,
    11 mantissa bits, subnormal step 2^-25, saturating at 2 - 2^-11), ties
    away from zero, from the format's definition."""
    x = x32.astype(np.float64)
    a = np.abs(x)
    e = np.floor(np.log2(np.maximum(a, 2.0 ** -14)))
    step = np.where(a < 2.0 ** -14, 2.0 ** -25, 2.0 ** (e - 11))
    r = np.minimum(np.floor(a / step + 0.5) * step, 2.0 - 2.0 ** -11)
    return np.sign(x) * r


def test_f16c_storage_encodes_to_nearest():
    g = (64, 4, 4)
    s = K.make_solver(K.case(g, None, omega1=1.0, u_in=0.0, faces=("periodic",) * 4), "f16c")
    rng = np.random.default_rng(5)
    w = O.weights()
    n = 64 * 16
    v = np.concatenate([rng.uniform(-1.9, 1.9, 27 * n // 3), rng.uniform(-1e-3, 1e-3, 27 * n // 3),
                        rng.uniform(-1e-6, 1e-6, 27 * n - 2 * (27 * n // 3))])
    v[:6] = [0.0, 2.5, -3.0, 2.0 ** -14, 2.0 ** -25 * 1.5, 1.0 + 2.0 ** -12]     # the last two are ties
    src = w[:, None] + v.reshape(27, n)
    s.set_pdfs(src.reshape(27, *g[::-1]))
    got = s.pdfs().reshape(27, n) - w[:, None]
    ref = f16c_round((src - w[:, None]).astype(np.float32))
    assert np.abs(got - ref).max() <= 1e-15


def test_degenerate_all_solid_and_empty_steps():
    g = (8, 4, 4)
    s = K.make_solver(K.case(g, np.ones(g[::-1], np.uint8)), "f32")
    s.step(0)
    s.step(3)
    s.sync()
    assert s.t == 3
    rho, u = s.macros()
    assert np.all(rho == 1) and np.all(u == 0)


# --------------------------------------------------------------------------
# conservation, instability flag, checkpoint, workspace ownership
# --------------------------------------------------------------------------
def test_periodic_totals_are_conserved():
    """Mass and momentum of a periodic box are invariants of the method.  The
    reference totals of the seeded state are exact sums (math.fsum) of the
    initial deviations; the drift bound is the rounding of 41 steps x 7680
    cells x 27 populations of size <~ 1e-2 in FP64."""
    import math
    c = K.case((24, 20, 16), None, omega1=1.9, faces=("periodic",) * 4, u_in=0.0, noise=(21, 1e-2))
    s = K.make_solver(c, "f64")
    t0 = s.totals()
    n = 24 * 20 * 16
    fbar = 1e-2 * I.pdf_noise(21, np.arange(n))
    cv = O.velocities()
    ref = [math.fsum(fbar.reshape(-1))] + [math.fsum((cv[:, d, None] * fbar).reshape(-1)) for d in range(3)]
    assert np.abs(t0 - np.array(ref)).max() < 1e-13
    s.step(41)
    t1 = s.totals()
    assert np.abs(t1 - t0).max() < 41 * n * 27 * 2.2e-16 * 1e-2


def test_instability_is_latched_and_steps_refused():
    from paper_2606_16765_gb300.lbm import LBMError, LBM_ERR_UNSTABLE, LBM_ERR_STATE
    c = K.case((16, 8, 8), None, omega1=1.9, faces=("periodic",) * 4, u_in=0.0, noise=(5, 0.2))
    s = K.make_solver(c, "f32")
    s.step(2)
    with pytest.raises(LBMError) as e:
        s.sync()
    assert e.value.status == LBM_ERR_UNSTABLE
    with pytest.raises(LBMError) as e2:
        s.step(1)
    assert e2.value.status == LBM_ERR_STATE
    s.macros()                               # reads still work


def test_checkpoint_resume_is_bitwise(tmp_path):
    d = I.sphere_channel_64()
    c = K.case(d["grid"], d["mask"], omega1=1.9, mean=(0, 1000, 2))
    a = K.make_solver(c, "f32", force_every=1)
    a.step(30)
    path = str(tmp_path / "ck.bin")
    a.save(path)
    a.step(31)
    b = K.make_solver(c, "f32", force_every=1)
    b.load(path)
    assert b.t == 30
    b.step(31)
    assert np.array_equal(a.pdfs(), b.pdfs())
    assert np.array_equal(a.mean()[0], b.mean()[0])
    assert np.array_equal(a.forces(), b.forces())


def test_library_owned_memory_matches_workspace():
    from paper_2606_16765_gb300 import lbm as B
    import torch
    d = I.sphere_channel_64()
    c = K.case(d["grid"], d["mask"], omega1=1.9, noise=(3, 1e-3))
    a = K.make_solver(c, "f32")
    p = B.make_params(storage="f32", omega1=1.9, u_in=0.05, faces=c["faces"])
    h = B.lbm_create(B.lbm_grid(*d["grid"]), d["mask"], p, torch.cuda.current_stream().cuda_stream)
    B.lbm_init_noise(h, 3, 1e-3)
    a.step(7)
    B.lbm_step(h, 7)
    out = np.zeros((27,) + a.shape)
    B.lbm_get_pdfs(h, out)
    B.lbm_destroy(h)
    assert np.array_equal(out, a.pdfs())


def test_argument_errors_are_reported():
    from paper_2606_16765_gb300.lbm import LBMError, Solver
    with pytest.raises(LBMError):
        Solver((8, 8, 8), faces=("outlet", "inlet", "wall", "wall"))
    with pytest.raises(LBMError):
        Solver((0, 8, 8))
    s = Solver((8, 8, 8), omega1=1.5)
    with pytest.raises(LBMError):
        s.step(-1)
    s.step(1)
    with pytest.raises(LBMError):            # set needs an even time step
        s.set_pdfs(np.zeros((27, 8, 8, 8)))


# --------------------------------------------------------------------------
# snapshots (full and half resolution) against oracle macros
# --------------------------------------------------------------------------
@pytest.mark.parametrize("halfres", [0, 1])
def test_snapshots(halfres):
    g = (33, 14, 12)
    mask = I.sphere(g, (10.0, 6.5, 5.5), 3.0)
    c = K.case(g, mask, omega1=1.8, noise=(31, 1e-3))
    s = K.make_solver(c, "f64", snap_first=3, snap_every=4, snap_count=3, snap_halfres=halfres)
    L = K.run_oracle(c, 0)
    want = {}
    for t in range(12):
        if t in (3, 7, 11):
            rho, u = L.macros()
            fld = np.concatenate([u, (rho[..., None] - 1) / 3], -1) * (mask == 0)[..., None]
            want[(t - 3) // 4] = O.halfres(fld) if halfres else fld
        L.step(1)
    s.step(12)
    for k, ref in want.items():
        got = s.snapshot(k)
        assert got.shape == ref.shape
        assert np.abs(got - ref).max() < 1e-6 * max(1.0, np.abs(ref).max())


# --------------------------------------------------------------------------
# 1024x512x512 channel (composite obstacle), launch configuration of the
# benchmark, on sampled cells that the oracle computes one by one from a
# neighbourhood of the seeded initial state
# --------------------------------------------------------------------------
def oracle_cell_after(mask, grid, faces, omega1, u_in, seed, amp, cell, steps, links=None):
    """The oracle on a box around `cell` large enough that nothing from its
    fake faces reaches the cell in `steps` steps (streaming moves one cell per
    step, the interpolated bounce-back reads two cells behind a link)."""
    nx, ny, nz = grid
    z, y, x = np.unravel_index(cell, (nz, ny, nx))
    R = 3 * steps + 1
    x0, x1 = max(0, x - R), min(nx, x + R + 1)
    y0, y1 = max(0, y - R), min(ny, y + R + 1)
    z0, z1 = max(0, z - R), min(nz, z + R + 1)
    sub = np.ascontiguousarray(mask[z0:z1, y0:y1, x0:x1])
    sg = (x1 - x0, y1 - y0, z1 - z0)
    zz, yy, xx = np.meshgrid(np.arange(z0, z1), np.arange(y0, y1), np.arange(x0, x1), indexing="ij")
    gcell = (xx + nx * (yy + ny * zz)).reshape(-1)
    w = O.weights()
    f = w[:, None] + amp * I.pdf_noise(seed, gcell)
    f[:, sub.reshape(-1) != 0] = w[:, None]
    sub_faces = ("inlet" if x0 == 0 else "wall", faces[1] if x1 == nx else "wall", "wall", "wall")
    p = O.params(*sg, omega1, u_in=u_in, faces=sub_faces)
    L = O.Lattice(p, sub)
    L.set_f(f.reshape(27, *sub.shape))
    if links is not None:                              # wall distances of the links inside the box
        lc, ld, lq = links
        X, Y, Z = lc % nx, (lc // nx) % ny, lc // (nx * ny)
        inside = (X >= x0) & (X < x1) & (Y >= y0) & (Y < y1) & (Z >= z0) & (Z < z1)
        qd = np.full((27, sg[0] * sg[1] * sg[2]), 0.5)
        local = (X[inside] - x0) + sg[0] * ((Y[inside] - y0) + sg[1] * (Z[inside] - z0))
        qd[ld[inside].astype(np.int64), local] = lq[inside]
        L.set_q(qd.reshape(27, sub.shape[0], sub.shape[1], sub.shape[2]))
    L.step(steps)
    return L.get_f()[:, z - z0, y - y0, x - x0]


@pytest.mark.parametrize("storage", ["f32", "f16c", "f16s"])
def test_full_size_channel_sampled_cells(storage):
    import torch
    d = I.composite_channel(0)
    grid, mask = d["grid"], d["mask"]
    nx, ny, nz = grid
    w1 = O.omega_from_re(d["re"], d["u_in"], d["l_ref"])
    from paper_2606_16765_gb300.lbm import Solver
    seed, amp = 77, 1e-3
    faces = ("inlet", "outflow", "wall", "wall")
    links = I.link_wall_distances(grid, d["obstacle"].prims, mask)
    s = Solver(grid, mask, storage=storage, omega1=w1, u_in=d["u_in"], faces=faces)
    s.set_wall_distances(links)
    s.init_noise(seed, amp)
    rng = np.random.default_rng(0)
    n = nx * ny * nz
    fluid_idx = np.flatnonzero(mask.reshape(-1) == 0)
    pick = list(rng.choice(fluid_idx, 120, replace=False))
    # cells next to the obstacle, on the inlet/outlet planes, walls and corners
    zz, yy, xx = np.nonzero(mask)
    for k in rng.choice(len(xx), 20, replace=False):
        for dx in (-1, 1):
            c = (xx[k] + dx) + nx * (yy[k] + ny * zz[k])
            if mask.reshape(-1)[c] == 0:
                pick.append(c)
    for (x, y, z) in [(0, 5, 7), (nx - 1, 100, 300), (0, 0, 0), (nx - 1, ny - 1, nz - 1),
                      (500, 0, 200), (700, ny - 1, 1), (3, 200, nz - 1), (nx - 1, 0, nz - 1)]:
        pick.append(x + nx * (y + ny * z))
    pick = np.array(sorted(set(int(p) for p in pick)), np.int64)
    # 16-bit: half an ulp is 2^-11 (binary16) or 2^-12 (F16C) of |fbar|
    # (<~ 3e-3 here); a few roundings per step
    tol = {"f32": 2e-7, "f16s": 8 * 2.0 ** -11 * 3e-3, "f16c": 8 * 2.0 ** -12 * 3e-3}[storage]
    for steps in (1, 2):
        s.step(1)
        got = s.cells(pick)
        for j, c in enumerate(pick):
            ref = oracle_cell_after(mask, grid, faces, w1, d["u_in"], seed, amp, c, steps, links)
            err = np.abs(got[j] - ref).max()
            assert err <= tol, (storage, steps, int(c), err)
    s.sync()
    del s
    torch.cuda.empty_cache()


# --------------------------------------------------------------------------
# interpolated bounce-back with wall distances
# --------------------------------------------------------------------------
QBB_CASES = {
    "sphere_outflow": ((37, 13, 11), [I.Primitive("sphere", (9.3, 6.2, 5.1), (6.6,))],
                       ("inlet", "outflow", "wall", "wall"), 1.8),
    "sphere_near_periodic_faces": ((20, 12, 10), [I.Primitive("sphere", (10.4, 1.3, 8.6), (7.0,))],
                                   ("periodic", "periodic", "periodic", "periodic"), 1.6),
    "torus_thin_gaps": ((30, 14, 12), [I.Primitive("torus", (12.2, 6.7, 5.4), (8.0, 2.2), 20.0)],
                        ("inlet", "outflow", "wall", "wall"), 1.9),
}


@pytest.mark.parametrize("name", sorted(QBB_CASES))
@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_interpolated_bounce_back_matches_oracle(name, storage):
    from paper_2606_16765_gb300.lbm import Solver
    g, prims, faces, w1 = QBB_CASES[name]
    mask = I.voxelize(g, prims)
    links = I.link_wall_distances(g, prims, mask)
    assert len(links[0]) > 0
    u_in = 0.0 if faces[0] == "periodic" else 0.05
    c = K.case(g, mask, omega1=w1, u_in=u_in, faces=faces, noise=(41, 2e-3))
    L = K.run_oracle(c, 0)
    L.set_q(I.dense_wall_distances(g, links))
    s = K.make_solver(c, storage, force_every=1)
    s.set_wall_distances(links)
    fluid = mask == 0
    for steps in (1, 1, 5, 13):
        s.step(steps)
        L.step(steps)
        err = np.abs(s.pdfs() - L.get_f())[:, fluid].max()
        assert err <= (1e-14 if storage == "f64" else 2e-7), (name, storage, L.t, err)
    F, Fr = s.forces(), L.forces()
    assert F.shape == Fr.shape
    ferr = np.abs(F - Fr).max() / max(np.abs(Fr).max(), 1e-30)
    print(f"qbb {name} {storage}: pdf err {err:.2e}, force err {ferr:.2e}")
    assert ferr <= (1e-12 if storage == "f64" else 1e-5)


def test_wall_distance_argument_errors():
    from paper_2606_16765_gb300.lbm import LBMError, Solver
    g = (16, 8, 8)
    prims = [I.Primitive("sphere", (7.3, 3.6, 4.1), (5.0,))]
    mask = I.voxelize(g, prims)
    s = Solver(g, mask, storage="f32", omega1=1.5)
    cell, d, q = I.link_wall_distances(g, prims, mask)
    with pytest.raises(LBMError):
        s.set_wall_distances((cell[:1], np.array([13], np.int8), q[:1]))        # rest direction
    with pytest.raises(LBMError):
        s.set_wall_distances((cell[:1], d[:1], np.array([1.5])))               # q out of range
    far = np.array([0], np.int64)                                             # a corner cell far from the sphere
    with pytest.raises(LBMError):
        s.set_wall_distances((far, np.array([26], np.int8), np.array([0.5])))
    s.set_wall_distances((cell, d, q))
    s.set_wall_distances((np.zeros(0, np.int64), np.zeros(0, np.int8), np.zeros(0)))   # back to halfway


# --------------------------------------------------------------------------
# fourth-order parametrisation with limiter (Sec. 3.2, Geier et al. 2017)
# --------------------------------------------------------------------------
def param4_cases():
    d = I.sphere_channel_64()
    yield "sphere channel 64x32x32, outflow, w1 1.95", K.case(
        d["grid"], d["mask"], omega1=1.95, u_in=0.05, faces=("inlet", "outflow", "wall", "wall"),
        noise=(51, 2e-3), param4=1, mean=(10, 60, 5))
    g = (29, 13, 11)
    yield "ragged periodic box, w1 1.9, large noise (limiter engaged)", K.case(
        g, I.sphere(g, (10.0, 6.0, 5.0), 2.5), omega1=1.9, u_in=0.0, faces=("periodic",) * 4,
        noise=(52, 5e-3), param4=1)
    yield "closed box, w1 1.85, bulk rate 1.3", K.case(
        (17, 9, 12), None, omega1=1.85, omega_bulk=1.3, u_in=0.0, faces=("wall",) * 4, noise=(53, 5e-3), param4=1)


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("which", [0, 1, 2])
def test_parametrised_collision_matches_oracle(storage, which):
    name, c = list(param4_cases())[which]
    L = K.run_oracle(c, 60)
    rho_r, u_r = L.macros()
    s = K.make_solver(c, storage)
    s.step(60)
    s.sync()
    rho, u = s.macros()
    fluid = c["mask"] == 0 if c["mask"] is not None else np.ones(rho.shape, bool)
    eu, er = K.rel_u_err(u, u_r, fluid), K.rho_err(rho, rho_r, fluid)
    print(f"param4 {name} {storage}: rel u err {eu:.3e} rho err {er:.3e}")
    tol = {"f64": 1e-12, "f32": 1e-5}[storage]
    assert eu <= tol and er <= tol
    if c["mean"][2]:
        m, ns = s.mean()
        mref, nref = L.means()
        assert ns == nref
        assert np.abs(m - mref)[fluid].max() / np.abs(mref[..., :3])[fluid].max() <= tol


def test_parametrisation_argument_errors():
    from paper_2606_16765_gb300.lbm import Solver, LBMError
    with pytest.raises(LBMError):
        Solver((8, 4, 4), None, omega1=1.0, omega_bulk=1.0, param4=1)   # undefined at omega1 = omega_bulk
    with pytest.raises(LBMError):
        Solver((8, 4, 4), None, omega1=1.9, param4=1, limiter=0.0)


# --------------------------------------------------------------------------
# monitor plane (Sec. 2: 2D snapshots of the centre x-y plane)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_monitor_plane_records_the_centre_plane_before_each_sampled_step(storage):
    """Planes of the sphere channel every 7 steps for 30 steps against the
    oracle's macros of the state before those steps at z = nz / 2, with a
    ring of 2 planes so that the host flush runs; a second plane position.
    The planes are recorded in FP32."""
    d = I.sphere_channel_64()
    nx, ny, nz = d["grid"]
    w1 = O.omega_from_re(d["re"], d["u_in"], d["l_ref"])
    c = K.case(d["grid"], d["mask"], omega1=w1, u_in=d["u_in"], faces=("inlet", "outflow", "wall", "wall"),
               noise=(61, 1e-3))
    for z in (-1, 3):
        s = K.make_solver(c, storage)
        s.set_plane_monitor(z=z, every=7, capacity=2)
        s.step(30)
        s.sync()
        planes, steps = s.plane_monitor()
        assert list(steps) == [0, 7, 14, 21, 28] and planes.shape == (5, ny, nx, 4)
        zz = nz // 2 if z < 0 else z
        L = K.run_oracle(c, 0)
        # the planes are FP32: FP64 storage is held to FP32 rounding
        tol = {"f64": 1e-6, "f32": 1e-5}[storage]
        for k, t in enumerate(steps):
            L.step(int(t) - L.t)
            rho, u = L.macros()
            ref = np.concatenate([u[zz], ((rho[zz] - 1) / 3)[..., None]], -1)
            ref[c["mask"][zz] != 0] = 0.0
            err = np.abs(planes[k] - ref).max() / np.abs(ref[..., :3]).max()
            assert err <= tol, (z, t, err)


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_inlet_outlet_cells_through_the_boundary_records(storage):
    """xface_edge = 1 (the batch members' setting): the inlet and outlet cells
    go through the boundary-cell records instead of the bulk kernel's face
    warps.  Same arithmetic per cell: the populations equal the default
    path's bitwise, and the oracle's within the storage's tolerance."""
    d = I.sphere_channel_64()
    w1 = O.omega_from_re(d["re"], d["u_in"], d["l_ref"])
    c = K.case(d["grid"], d["mask"], omega1=w1, u_in=d["u_in"], faces=("inlet", "outflow", "wall", "wall"),
               noise=(71, 1e-3))
    L = K.run_oracle(c, 40)
    rho_r, u_r = L.macros()
    a = K.make_solver(c, storage, xface_edge=1)
    b = K.make_solver(c, storage)
    a.step(40)
    b.step(40)
    a.sync()
    b.sync()
    assert a.info().edge_cells > b.info().edge_cells
    assert np.array_equal(a.pdfs(), b.pdfs())
    rho, u = a.macros()
    fl = c["mask"] == 0
    tol = {"f64": 1e-12, "f32": 1e-5}[storage]
    assert K.rel_u_err(u, u_r, fl) <= tol and K.rho_err(rho, rho_r, fl) <= tol
