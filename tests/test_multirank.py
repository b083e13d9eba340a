"""The N > 1 path of bench.py on CPU: two gloo ranks agree on the slowest
rank's time, report the whole-job rate over both ranks' work, fit distinct
workloads, and only rank 0 runs the oracle arm."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(world),
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench.rank_env()
        ms = bench.max_over_ranks(10.0 + 5.0 * r, w)          # rank 1 is the slower one
        rate = bench.whole_job_rate(1000, w, ms)
        seeds = [None] * w
        dist.all_gather_object(seeds, bench.rank_seed(r))
        ref = bench.run_reference(type("A", (), {"steps": 1, "warmup": 0, "gpus": w})()) if r != 0 else "skip"
        out[rank] = (w, r, local, ms, rate, tuple(seeds), ref)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    for rank in range(world):
        w, r, local, ms, rate, seeds, ref = out[rank]
        assert (w, r, local) == (2, rank, rank)
        assert ms == 15.0                                       # max over ranks, on every rank
        assert rate == pytest.approx(2 * 1000 / 15e-3)          # both ranks' units / slowest time
        assert len(set(seeds)) == 2                             # distinct workloads per rank
        if rank != 0:
            assert ref is None                                  # the oracle arm runs on rank 0 only
