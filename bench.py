#!/usr/bin/env python
"""Throughput of the fused D3Q27 cumulant LBM step on the full-size channel.

Workload: 1024x512x512 channel (268M cells) with a seeded composite obstacle
(2-4 random primitives), Re = 10^4 on the channel height, inlet u = 0.05;
shifted pdfs in FP32 (headline) and FP16 (reported beside it).  A step is one
full time step of the hot path: fused stream + collide over all fluid cells
with the obstacle force recorded every step, the FP64 time average sampled
every 10 steps, and 20 half-resolution snapshots 25 steps apart at the end of
the timed window.

Default run: python bench.py [--steps K] [--warmup W].  Under torchrun with
N > 1 each rank runs its own replica of the workload (independent problems;
no collective on the data path) and rank 0 prints the aggregate.
--impl reference times the FP64 CPU oracle on the host cores instead.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS & % HBM roofline (D3Q27); FNO mean-field speedup vs LBM at ≤5% rel L2"
NOMINAL_HBM_GBS = 8000.0
BYTES_PER_POP = {"f64": 8, "f32": 4, "f16s": 2, "bf16s": 2, "f16c": 2}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_hash():
    """Hash of the LBM kernel sources (the FNO sources do not enter)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2606_16765_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name.startswith("lbm") and name.endswith((".cu", ".cuh", ".h")):
            h.update(open(os.path.join(csrc, name), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel, workload):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        recs = json.load(open(path))
    except Exception:
        return None
    src = kernel_source_hash()
    for r in recs:
        if r.get("kernel") == kernel and r.get("workload") == workload and r.get("source_hash") == src:
            return r.get("bytes_per_launch")
    return None


def recorded_instructions(kernel):
    """Warp instructions per interior cell of a bulk kernel from a committed
    ncu summary (profiles/alu.json), if it was taken on the current kernel
    sources; the count does not depend on the grid size."""
    path = os.path.join(ROOT, "profiles", "alu.json")
    if not os.path.exists(path):
        return None
    try:
        recs = json.load(open(path))
    except Exception:
        return None
    src = kernel_source_hash()
    for r in recs:
        if r.get("kernel") == kernel and r.get("source_hash") == src:
            return r.get("warp_instructions_per_cell")
    return None


def sm_count():
    """Multiprocessor count of the current device (cudaDevAttrMultiProcessorCount)."""
    import torch
    return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)


def alu_roofline(kernel, cells, ms, clocks, sms):
    """Issue-rate roofline of a bulk kernel: achieved warp instructions per
    second against `sms` SMs (read from the device) x 4 schedulers x 1 warp
    instruction per clock at the SM clock sampled during the run."""
    ipc = recorded_instructions(kernel)
    if ipc is None or not clocks:
        return None
    achieved = ipc * cells / (ms / 1e3)
    peak = sms * 4 * clocks["sm_mhz"] * 1e6
    return {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "T warp-instructions/s",
            "frac": achieved / peak, "warp_instructions_per_cell": ipc, "kernel": kernel,
            "peak_source": f"{sms} SMs (device attribute) x 4 issue slots x sampled SM clock"}


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# distributed helpers (replicas; only timing and unit counts are exchanged)
# ---------------------------------------------------------------------------
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate(ms, units, ws, backend_ready):
    """Max time over ranks and total units (the job's throughput)."""
    if ws == 1 or not backend_ready:
        return ms, units
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    u = torch.tensor([units], dtype=torch.float64, device=t.device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------
def workload(grid):
    """The composite channel and the wall distances of its obstacle links
    (interpolated bounce-back), computed on the host before any timing."""
    from paper_2606_16765_gb300 import inputs as I
    d = I.composite_channel(0, grid=grid)
    d["links"] = I.link_wall_distances(d["grid"], d["obstacle"].prims, d["mask"])
    return d


def schedule(steps, warmup):
    """Epilogue schedule over the timed window [warmup, warmup + steps)."""
    nsnap = min(20, max(1, steps // 25))
    # the last snapshot at the last timed step, the others 25 steps apart before it
    return dict(mean_start=warmup, mean_end=warmup + steps, mean_every=10,
                snap_first=warmup + steps - 1 - 25 * (nsnap - 1), snap_every=25, snap_count=nsnap,
                snap_halfres=1, force_every=1)


def epilogue_counts(sch, warmup, steps):
    """Snapshots, mean samples and force rows that fall inside the timed
    window [warmup, warmup + steps) under the schedule `sch`."""
    lo, hi = warmup, warmup + steps
    snaps = [sch["snap_first"] + k * sch["snap_every"] for k in range(sch["snap_count"])]
    means = range(sch["mean_start"], sch["mean_end"], sch["mean_every"])
    return {"snapshots": sum(1 for t in snaps if lo <= t < hi),
            "mean_samples": sum(1 for t in means if lo <= t < hi),
            "force_rows": len(range(lo, hi, sch["force_every"]))}


def run_ours(args, storage, d, ws, device_index, param4=0):
    import torch
    from paper_2606_16765_gb300.lbm import Solver

    K, W = args.steps, args.warmup
    sch = schedule(K, W)
    s = Solver(d["grid"], d["mask"], storage=storage, re=d["re"], u_in=d["u_in"], l_ref=d["l_ref"],
               block_x=args.block_x, param4=param4, **sch)
    s.set_wall_distances(d["links"])
    info = s.info()
    s.step(W)
    s.sync()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.timing(True)
    s.timing_read(reset=True)
    launches0 = s.info().launches
    clocks = ClockSampler(device_index)
    barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    e0.record(stream)
    s.step(K)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    s.sync()
    rep = s.timing_read(reset=True)
    launches = s.info().launches - launches0
    res = dict(ms=ms, info=info, rep=rep, clocks=clk, launches=launches, storage=storage)
    s.close()
    del s
    torch.cuda.empty_cache()
    return res


def run_e2e(args, storage, d):
    """Through the C ABI with host buffers: mask upload, K steps, half-res
    mean read-back, all inside the timed region."""
    import numpy as np
    import torch
    from paper_2606_16765_gb300 import lbm as B

    K = args.steps
    p = B.make_params(storage=storage, re=d["re"], u_in=d["u_in"], l_ref=d["l_ref"],
                      block_x=args.block_x, **schedule(K, 0))
    grid = B.lbm_grid(*d["grid"])
    nx, ny, nz = d["grid"]
    mean = np.zeros((((nz + 1) // 2), ((ny + 1) // 2), ((nx + 1) // 2), 4), np.float32)
    mask = np.ascontiguousarray(d["mask"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h = B.lbm_create(grid, mask, p, torch.cuda.current_stream().cuda_stream)
    B.lbm_set_wall_distances(h, *d["links"])
    B.lbm_sync(h)
    t1 = time.perf_counter()
    B.lbm_step(h, K)
    B.lbm_sync(h)
    t2 = time.perf_counter()
    B.lbm_read_mean(h, mean, 1, 1)
    t3 = time.perf_counter()
    info = B.lbm_get_info(h)
    B.lbm_destroy(h)
    torch.cuda.empty_cache()
    link_bytes = sum(a.nbytes for a in d["links"])
    return dict(seconds=t3 - t0, fluid=info.fluid_cells, h2d=mask.nbytes + link_bytes, d2h=mean.nbytes,
                split={"create_upload_s": t1 - t0, "step_s": t2 - t1, "readback_s": t3 - t2})


def run_batch(steps, warmup, storage="f16s", n=32):
    """32 seeded channels on uneven grids {128,192,256} x {64,96,128}^2, Re
    log-uniform in [1e3, 1e4] on the channel height, stepped together by the
    batched driver (graph-captured chunks, autotuned block shape), with the
    FP64 time average every 10 steps and the obstacle force every step."""
    import torch
    from paper_2606_16765_gb300 import inputs as I
    from paper_2606_16765_gb300.lbm import Batch

    chans = I.batch_channels(0, n=n)
    total = warmup + steps + 40
    ms = []
    for d in chans:
        ms.append(dict(grid=d["grid"], mask=d["mask"], storage=storage, re=d["re"], u_in=d["u_in"],
                       l_ref=d["l_ref"], mean_start=0, mean_end=10 ** 9, mean_every=10,
                       force_every=1, force_capacity=total + 64))
    b = Batch(ms)
    for g, d in enumerate(chans):
        b.set_wall_distances(g, I.link_wall_distances(d["grid"], d["obstacle"].prims, d["mask"]))
    bx, by, tune_ms = b.autotune(trials=2)
    b.run(warmup)
    b.sync()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    i0 = b.info()
    torch.cuda.synchronize()
    e0.record(stream)
    b.run(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    b.sync()
    i1 = b.info()
    t = e0.elapsed_time(e1)
    ups = i1.lattice_updates - i0.lattice_updates
    cells = sum(int((d["mask"] == 0).sum()) for d in chans)
    out = {"value": ups / (t / 1e3) / 1e6, "unit": "MLUPS", "storage": storage, "members": n,
           "fluid_cells": cells, "steps": int(i1.t - i0.t), "ms_per_step": t / max(1, i1.t - i0.t),
           "block": [bx, by], "graph_captures": int(i1.graph_captures),
           "graph_launches": int(i1.graph_launches - i0.graph_launches),
           "gpu_launches": int(i1.kernel_launches - i0.kernel_launches),
           "bytes_per_update": 54 * BYTES_PER_POP[storage]}
    out["hbm_gbs"] = out["value"] * 1e6 * out["bytes_per_update"] / 1e9
    b.close()
    torch.cuda.empty_cache()
    return out


def fno_algorithmic_bytes(batch, n, width=32, cin=4, cout=4, layers=4, act=2):
    """Bytes an FNO forward and a training step must move at least, the
    activations each written once and read once: FP32 input and output,
    BF16 (act = 2 B) activations of `width` channels.  Forward: input, lift
    output, per layer read v and write v', projection read v_L, output.
    Training adds the stored pre-activations (written in the forward, read in
    the backward), per layer the layer input re-read and an FP32 gradient
    read and written, and the projection and lift backward (v_L, x, the
    output gradient read, FP32 input gradients written)."""
    cells = batch * n
    io_in, io_out = cells * cin * 4, cells * cout * 4
    a = cells * width * act
    g = cells * width * 4
    fwd = io_in + a + layers * 2 * a + a + io_out
    train = fwd + layers * a + layers * (a + a + 2 * g) + (a + io_out + g) + (io_in + g)
    return fwd, train


def run_fno(batch=8, reps=10):
    """FNO surrogate at 128x64x64 (4 Fourier layers, width 32, modes 16x8x8,
    BF16 activations, tensor-core mode contraction): forward and training-step
    time for a batch of 8 with inputs resident, and the LBM run it replaces
    (one held-out geometry of the surrogate's data set alone to 15
    flow-through times, CUDA events).  Prediction accuracy comes from the
    trained pipeline (paper_2606_16765_gb300.fno_pipeline), not from here."""
    from paper_2606_16765_gb300 import fno_pipeline as P

    r = P.time_fno(batch=batch, reps=reps)
    t_lbm = P.time_lbm_to_end(P.sample(2000))
    fwd = r["forward_ms_per_batch"]
    nx, ny, nz = P.GRID
    b_fwd, b_train = fno_algorithmic_bytes(batch, nx * ny * nz)
    peak, kind = measured_peaks()
    roof = {"bound": "hbm", "unit": "GB/s", "peak": peak, "peak_source": kind,
            "bytes_per_forward": b_fwd, "bytes_per_train_step": b_train,
            "achieved": b_fwd / (fwd / 1e3) / 1e9, "frac": b_fwd / (fwd / 1e3) / 1e9 / peak,
            "train_achieved": b_train / (r["train_step_ms"] / 1e3) / 1e9,
            "train_frac": b_train / (r["train_step_ms"] / 1e3) / 1e9 / peak,
            "note": "algorithmic bytes: each activation written once and read once (BF16), FP32 input/output "
                    "and gradients; the implementation's unfused stages move more"}
    return {"grid": list(P.GRID), "batch": batch, "forward_ms_per_batch": fwd, "roofline": roof,
            "forward_ms_per_sample": fwd / batch, "train_step_ms": r["train_step_ms"],
            "train_samples_per_s": batch / (r["train_step_ms"] / 1e3), "lbm_15ft_seconds_one_sample": t_lbm,
            "speedup_vs_lbm": t_lbm / (fwd / batch / 1e3), "dtype": "bf16 activations, fp32 accumulation"}


def oracle_sub_box(O, d, bx, by, bz):
    """FP64 oracle lattice on a bx x by x bz sub-box of the channel around the
    obstacle, with the GPU arm's boundary set: moving-wall inlet, convective
    outflow, no-slip lateral walls and the interpolated bounce-back on the
    sub-box's obstacle links (wall distances of the shifted primitives)."""
    import dataclasses
    import numpy as np
    from paper_2606_16765_gb300 import inputs as I
    nx, ny, nz = d["grid"]
    bx, by, bz = min(bx, nx), min(by, ny), min(bz, nz)
    x0 = max(0, min(nx - bx, int(0.3 * nx) - bx // 3))
    y0, z0 = (ny - by) // 2, (nz - bz) // 2
    sub = np.ascontiguousarray(d["mask"][z0:z0 + bz, y0:y0 + by, x0:x0 + bx])
    prims = [dataclasses.replace(pr, center=(pr.center[0] - x0, pr.center[1] - y0, pr.center[2] - z0))
             for pr in d["obstacle"].prims]
    w1 = O.omega_from_re(d["re"], d["u_in"], d["l_ref"])
    L = O.Lattice(O.params(bx, by, bz, w1, u_in=d["u_in"], faces=("inlet", "outflow", "wall", "wall")), sub)
    links = I.link_wall_distances((bx, by, bz), prims, sub)
    if len(links[0]):
        L.set_q(I.dense_wall_distances((bx, by, bz), links))
    return L, sub, (bx, by, bz), len(links[0])


def cpu_baseline(d, seconds=12.0, box=(128, 96, 96)):
    """FP64 oracle on the host cores, on a sub-box of the same channel around
    the obstacle, stepped until ~`seconds` of CPU work."""
    import numpy as np
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    import oracle.lbm as O
    L, sub, (bx, by, bz), nq = oracle_sub_box(O, d, *box)
    fluid = int((sub == 0).sum())
    steps, t0 = 0, time.perf_counter()
    while True:
        L.step(1)
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds or steps >= 200:
            break
    return {"value": fluid * steps / el / 1e6, "unit": "MLUPS", "cores": int(os.environ["OMP_NUM_THREADS"]),
            "kind": "oracle",
            "sample": f"{bx}x{by}x{bz} sub-box of the channel around the obstacle, {steps} FP64 steps, {el:.1f} s; "
                      f"inlet, convective outflow, walls, interpolated bounce-back on {nq} links"}


def reference_arm(args):
    """The FP64 CPU oracle timed on the host cores, each step a bounded
    sample of the workload sized so that W + K steps take ~100 s."""
    import numpy as np
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    import oracle.lbm as O
    grid = tuple(int(v) for v in args.grid.split(","))
    d = workload(grid)
    nx, ny, nz = grid
    w1 = O.omega_from_re(d["re"], d["u_in"], d["l_ref"])
    # calibrate the per-cell cost on a small box
    cal = O.Lattice(O.params(32, 16, 16, w1, u_in=d["u_in"]))
    t0 = time.perf_counter()
    cal.step(2)
    per_cell = (time.perf_counter() - t0) / (2 * 32 * 16 * 16)
    budget = 100.0 / max(1, args.steps + args.warmup)
    cells = max(16 * 8 * 8, min(nx * ny * nz, int(budget / per_cell)))
    a = max(8, int(round((cells / 2) ** (1 / 3))))
    L, sub, (bx, by, bz), nq = oracle_sub_box(O, d, 2 * a, a, a)
    fluid = int((sub == 0).sum())
    L.step(args.warmup)
    t0 = time.perf_counter()
    L.step(args.steps)
    el = time.perf_counter() - t0
    v = fluid * args.steps / el / 1e6
    sample = (f"{bx}x{by}x{bz} sub-box of the channel around the obstacle per step; inlet, convective outflow, "
              f"walls, interpolated bounce-back on {nq} links")
    line = {
        "metric": METRIC, "value": v, "unit": "MLUPS", "impl": "reference", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_block(grid, "f64", None),
        "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": int(os.environ["OMP_NUM_THREADS"]),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_block(grid, storage, info, counts=None):
    nx, ny, nz = grid
    if counts is None:
        epi = "obstacle force every step, FP64 mean every 10 steps, half-res snapshots 25 steps apart"
    else:
        epi = (f"obstacle force every step ({counts['force_rows']} rows), FP64 mean every 10 steps "
               f"({counts['mean_samples']} samples), {counts['snapshots']} half-res snapshots 25 steps apart "
               f"in the timed window")
    c = {"workload": f"composite-obstacle channel {nx}x{ny}x{nz}, Re=1e4 on the channel height, u_in=0.05, seed 0",
         "grid": [nx, ny, nz], "storage": storage,
         "epilogues": epi,
         "boundaries": "moving-wall velocity inlet, convective extrapolation outflow, no-slip walls, "
                       "interpolated (quadratic) bounce-back on the obstacle links",
         "l2": "inputs larger than L2 (pdf array >> 129 MB), no flush"}
    if info is not None:
        c.update(fluid_cells=int(info.fluid_cells), bulk_cells=int(info.bulk_cells),
                 interior_cells=int(info.interior_cells), edge_cells=int(info.edge_cells),
                 block_x=int(info.block_x))
    return c


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--storage", default="f32", choices=["f32", "f16s", "f16c", "bf16s", "f64"])
    ap.add_argument("--also", default="f16s,f16c,f32+param4",
                    help="comma list of extra storages to report, '+param4' for the fourth-order "
                         "parametrised collision ('' for none)")
    ap.add_argument("--grid", default="1024,512,512")
    ap.add_argument("--block-x", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--batch-members", type=int, default=32,
                    help="channels of the batch leg (32 is the batched configuration; fewer for small captures)")
    ap.add_argument("--no-fno", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        reference_arm(args)
        return

    import torch
    ws, rank, local = dist_env()
    backend = False
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
        backend = True
    else:
        torch.cuda.set_device(0)
    from paper_2606_16765_gb300 import _build
    if rank == 0:
        _build.build()
    barrier(ws)

    grid = tuple(int(v) for v in args.grid.split(","))
    d = workload(grid)
    res = run_ours(args, args.storage, d, ws, local)
    counts = epilogue_counts(schedule(args.steps, args.warmup), args.warmup, args.steps)
    info, rep = res["info"], res["rep"]
    K = args.steps
    ms, units = aggregate(res["ms"], float(info.fluid_cells) * K, ws, backend)
    mlups = units / (ms / 1e3) / 1e6

    peak, peak_kind = measured_peaks()
    sms = sm_count()
    s_b = BYTES_PER_POP[args.storage]
    # dominant kernel: the bulk kernel of odd steps without epilogue
    kind = 1 if rep.bulk_n[1] > 0 else 0
    bulk_ms = rep.bulk_ms[kind] / max(1, rep.bulk_n[kind])
    bytes_launch = 54 * s_b * info.interior_cells
    achieved = bytes_launch / (bulk_ms / 1e3) / 1e9
    kname = f"k_step_bulk<{args.storage},odd={bool(kind & 1)},epi=False>"
    traffic = recorded_traffic(kname, "composite channel %dx%dx%d" % grid)
    per_kind = {}
    for k, nm in enumerate(["even", "odd", "even+epilogue", "odd+epilogue"]):
        if rep.bulk_n[k]:
            t = rep.bulk_ms[k] / rep.bulk_n[k]
            per_kind[nm] = {"launches": int(rep.bulk_n[k]), "ms": t,
                            "gbs": 54 * s_b * info.interior_cells / (t / 1e3) / 1e9}
    edge_ms = rep.edge_ms / max(1, rep.steps)

    line = {
        "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": ws, "steps": K, "warmup": args.warmup,
        "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.storage == "f64" else "f32", "data": "synthetic",
        "config": config_block(grid, args.storage, info, counts),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_source": peak_kind,
                     "kernel": kname, "scope": "bulk kernel only (odd step, no epilogue)",
                     "bytes_per_launch": bytes_launch,
                     "frac_of_nominal_8000": achieved / NOMINAL_HBM_GBS},
        "step_roofline": {"scope": "whole step (bulk + edge + between-step kernels + epilogues): "
                                   "fluid MLUPS x pdf bytes per update",
                          "achieved": mlups * 1e6 * 54 * s_b / 1e9, "peak": peak, "unit": "GB/s",
                          "frac": mlups * 1e6 * 54 * s_b / 1e9 / peak / max(1, ws)},
        "sm_count": sms,
        "alu_roofline": alu_roofline(kname, info.interior_cells, bulk_ms, res["clocks"], sms),
        "kernels": {"bulk": per_kind, "edge_ms_per_launch": edge_ms},
        "gpu_launches": int(res["launches"]),
        "clocks": res["clocks"],
    }
    if rank == 0:
        for extra_name in [e for e in args.also.split(",") if e and e != args.storage]:
            extra, p4 = (extra_name.split("+")[0], 1) if extra_name.endswith("+param4") else (extra_name, 0)
            r2 = run_ours(args, extra, d, 1, local, param4=p4)
            b2 = 54 * BYTES_PER_POP[extra]
            k2 = 1 if r2["rep"].bulk_n[1] > 0 else 0
            t2 = r2["rep"].bulk_ms[k2] / max(1, r2["rep"].bulk_n[k2])
            line.setdefault("other_storage", {})[extra_name] = {
                "value": float(r2["info"].fluid_cells) * K / (r2["ms"] / 1e3) / 1e6, "unit": "MLUPS",
                "ms_per_step": r2["ms"] / K,
                "interior_kernel_gbs": b2 * r2["info"].interior_cells / (t2 / 1e3) / 1e9,
                "interior_kernel_frac": b2 * r2["info"].interior_cells / (t2 / 1e3) / 1e9 / peak,
                "alu_roofline": (None if p4 else
                                 alu_roofline(f"k_step_bulk<{extra},odd={bool(k2 & 1)},epi=False>",
                                              r2["info"].interior_cells, t2, r2["clocks"], sms)),
                "collision": "fourth-order parametrisation with limiter (Sec. 3.2)" if p4 else "plain cumulant",
                "clocks": r2["clocks"]}
        if not args.no_batch:
            line["batch"] = run_batch(args.steps, 20, n=args.batch_members)
        if not args.no_fno:
            line["fno"] = run_fno()
        if not args.no_e2e:
            e = run_e2e(args, args.storage, d)
            line["e2e"] = {"value": e["fluid"] * K / e["seconds"] / 1e6, "unit": "MLUPS",
                           "h2d_bytes_per_step": e["h2d"] / K, "d2h_bytes_per_step": e["d2h"] / K,
                           "seconds": e["seconds"], "split_seconds": e["split"],
                           "note": "create+upload covers the device allocation of the 29 GB pdf array, "
                                   "the mask and link upload and the cell classification"}
        if ws == 1 and not args.no_cpu:
            line["cpu_baseline"] = cpu_baseline(d)
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
