"""The N > 1 path of the benchmark on CPU: two gloo ranks, each solving its
own transmitter (weak scaling, no collective in the data path), joined only
by the max-over-ranks timing.  Runs without a GPU."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
import paper_2304_00233_b300 as emm
from paper_2304_00233_b300 import workloads as W


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl = W.marine_1d()
        src = bench.rank_source(wl.src, rank)
        # the rank's transmitter lies on the grid, outside the CPML, with the
        # same 4th-order stencil on every rank (host-side locate, no GPU)
        grid = emm.grid_for(wl)
        start, w = grid.locate(0, src)
        t = 1.0 + 0.5 * rank                      # this rank's "duration"
        slow = bench.max_over_ranks(t, dist, "cpu")
        out[rank] = (float(src[0]), slow, [int(v) for v in start])
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_sources_and_take_the_max_time():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    x0, x1 = res[0][0], res[1][0]
    assert x1 - x0 == pytest.approx(bench.TOW_SPACING)          # distinct transmitters
    assert res[0][1] == res[1][1] == pytest.approx(1.5)          # both see the slowest rank
    assert res[0][2] != res[1][2]                                # different stencils


def test_aggregate_rate_counts_every_rank():
    one = bench.aggregate_rate(1, 3_411_720, 6934, 5, 3.0)
    assert bench.aggregate_rate(8, 3_411_720, 6934, 5, 3.0) == pytest.approx(8 * one)
    assert bench.max_over_ranks(2.5) == 2.5


def test_eight_rank_sources_stay_on_the_grid():
    wl = W.marine_1d()
    grid = emm.grid_for(wl)
    for rank in range(8):
        grid.locate(0, bench.rank_source(wl.src, rank))    # raises on EMM_EOUTSIDE
