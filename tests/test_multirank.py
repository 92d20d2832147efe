"""The multi-process path of the benchmark on the CPU: two gloo ranks on
127.0.0.1.  Views are independent, so each rank renders its own view of the
replicated scene with no collective in the step; only the job's time (the
slowest rank's) is reduced, and rank 0 reports views over that time."""
import io
import os
import socket
from contextlib import redirect_stdout

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, results):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench.rank_env()
        ms_local = 2.0 + 0.5 * r  # rank 1 is the slower one
        ms_max = bench.max_over_ranks(ms_local, w, dist)
        results[r] = (w, r, local, bench.rank_azimuth(r), ms_max, bench.job_ms_per_view(ms_max, w))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_the_job_time():
    world = 2
    with mp.Manager() as mgr:
        results = mgr.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), results), nprocs=world, join=True)
        res = dict(results)
    assert sorted(res) == [0, 1]
    for r, (w, rr, local, az, ms_max, per_view) in res.items():
        assert (w, rr, local) == (2, r, r)
        assert ms_max == 2.5                # the slowest rank sets the step time
        assert per_view == 2.5 / 2          # two views per step over the job
    assert res[0][3] != res[1][3]           # each rank has its own view
    assert res[0][3] == bench.rank_azimuth(0) == -90.0


def test_single_process_defaults(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.rank_env() == (1, 0, 0)
    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.job_ms_per_view(3.0, 1) == 3.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    """Under torchrun every rank but 0 leaves without work or output."""
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    args = bench.parse(["--impl", "reference"])
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args)
    assert buf.getvalue() == ""
