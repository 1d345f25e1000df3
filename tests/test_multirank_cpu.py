"""The multi-rank bookkeeping of bench.py on CPU: two gloo ranks draw
different scenario sets (weak scaling) and combine their timings as max
elapsed time and total converged instances.  No data exchange is needed by
the solver itself: instances are independent."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import gridgen
    g = gridgen.make_grid("mesh30_b64")
    sc = bench.rank_scenarios("mesh30_b64", g, rank, batch=8)
    ms, conv = bench.combine_ranks(10.0 + rank, 8 - rank, torch.device("cpu"))
    # a tiny oracle solve per rank: every rank's instances converge on their own
    from oracle import nrpf
    Y = nrpf.make_ybus(g.n, g.f, g.t, g.r, g.x, g.b)
    _, it, st = nrpf.newton_batch(Y, sc.sbus(g)[:2], sc.v0_flat(g)[:2], g.bus_type)
    out[rank] = (ms, conv, float(sc.factors[0, 0]), int(np.sum(st == 0)))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_gloo_ranks_weak_scaling():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        out = man.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    assert res[0][0] == res[1][0] == 11.0          # max elapsed over ranks
    assert res[0][1] == res[1][1] == 15.0          # total converged: 8 + 7
    assert res[0][2] != res[1][2]                  # different scenario draws per rank
    assert res[0][3] == res[1][3] == 2
