"""The N > 1 path of the benchmark on CPU: two gloo ranks, each solving its
own transmitter (weak scaling, no collective during the solve), joined by
the max-over-ranks timing, the gather of the receiver arrays on rank 0 and
the sum of the per-transmitter gradients of a sharded survey.  Runs without
a GPU."""
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
        # the end of a survey: receiver arrays gathered on rank 0, the
        # per-transmitter gradient volumes of each rank's share summed
        G = torch.full((3, 6, 2), complex(rank + 1, -rank), dtype=torch.complex128)
        got = bench.gather_to_rank0(G, dist, world)
        mine = bench.shard(list(range(8)), rank, world)
        g = torch.zeros(4, 5, dtype=torch.float64)
        for k in mine:                           # one "gradient" per transmitter
            g += float(k + 1)
        bench.sum_over_ranks(g, dist)
        out[rank] = (float(src[0]), slow, [int(v) for v in start],
                     None if got is None else got.numpy(), mine, g.numpy())
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
    # rank 0 holds every rank's receiver arrays, in rank order
    assert res[1][3] is None
    assert res[0][3].shape == (2, 3, 6, 2)
    assert np.all(res[0][3][0] == 1.0) and np.all(res[0][3][1] == 2.0 - 1.0j)
    # the transmitters are shared out without overlap; the summed gradient is
    # that of all eight on both ranks
    assert sorted(res[0][4] + res[1][4]) == list(range(8)) and not set(res[0][4]) & set(res[1][4])
    assert np.all(res[0][5] == sum(range(1, 9))) and np.all(res[1][5] == res[0][5])


def test_aggregate_rate_counts_every_rank():
    one = bench.aggregate_rate(1, 3_411_720, 6934, 5, 3.0)
    assert bench.aggregate_rate(8, 3_411_720, 6934, 5, 3.0) == pytest.approx(8 * one)
    assert bench.max_over_ranks(2.5) == 2.5
    t = torch.ones(3)
    assert bench.sum_over_ranks(t) is t and bench.gather_to_rank0(t).shape == (1, 3)
    assert bench.shard(list(range(8)), 0, 1) == list(range(8))


def test_eight_rank_sources_stay_on_the_grid():
    wl = W.marine_1d()
    grid = emm.grid_for(wl)
    for rank in range(8):
        grid.locate(0, bench.rank_source(wl.src, rank))    # raises on EMM_EOUTSIDE
