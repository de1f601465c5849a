"""The multi-process path of bench.py (N replicas, one per GPU, no collective
on the data path): the job's time is the maximum over ranks, its units the
sum, and the barrier holds every rank.  World size 2 over gloo on the CPU."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import json
    import sys

    import torch.distributed as dist

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    ws, r, local = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=ws)
    bench.barrier(ws)
    ms, units = bench.aggregate(10.0 + 5.0 * r, 1000.0 * (r + 1), ws, True)
    bench.barrier(ws)
    with open(os.path.join(out_dir, f"rank{r}.json"), "w") as fp:
        json.dump(dict(ws=ws, rank=r, local=local, ms=ms, units=units), fp)
    dist.destroy_process_group()


def test_two_replicas_take_the_max_time_and_the_summed_units(tmp_path):
    import json

    import torch.multiprocessing as mp

    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for r, d in enumerate(res):
        assert d["ws"] == 2 and d["rank"] == r and d["local"] == r
        assert d["ms"] == pytest.approx(15.0)          # slowest rank
        assert d["units"] == pytest.approx(3000.0)     # all ranks' work


def test_single_process_needs_no_backend():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.aggregate(7.0, 11.0, 1, False) == (7.0, 11.0)
