"""Host logic of bench.py's N > 1 path: one replica per rank, no data-path
collective, the job time is the slowest rank's and the job rate sums all
ranks' cell-updates.  Runs as world-size-2 gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, lr = bench.replica_layout()
        ms_local = 10.0 + 5.0 * r          # rank 1 is the slower one
        ms = bench.max_over_ranks(torch, ms_local, dist, "cpu")
        rate = bench.whole_job_rate(1000, w, 4, ms)
        q.put((r, lr, w, ms, rate))
    finally:
        dist.destroy_process_group()


def test_layout_defaults_to_one_gpu():
    assert bench.replica_layout({}) == (1, 0, 0)
    assert bench.replica_layout({"WORLD_SIZE": "4", "RANK": "2", "LOCAL_RANK": "2"}) == (4, 2, 2)


def test_single_rank_keeps_its_time():
    assert bench.max_over_ranks(torch, 3.5, None, "cpu") == 3.5
    assert bench.whole_job_rate(1000, 1, 4, 2.0) == pytest.approx(2.0e6)


def test_two_gloo_ranks_take_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    for r, lr, w, ms, rate in out:
        assert lr == r and w == 2
        assert ms == 15.0                                  # max over ranks
        assert rate == pytest.approx(1000 * 2 * 4 / 15e-3)  # all ranks' cells, slowest time
