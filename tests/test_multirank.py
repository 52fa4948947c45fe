"""Two gloo ranks on CPU exercise bench.py's multi-rank logic: each rank gets
its own design seed and the timed region is reduced by max over ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2604_25728_gb300 import workloads as wl
    w = wl.mid()
    seed = bench.rank_seed(rank)
    b = wl.phase_indices(seed, w.M, w.N, w.B)
    t = bench.max_over_ranks(1.5 + rank, "cpu")
    out[rank] = (seed, int(b.sum()), t)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_get_distinct_designs_and_max_timing():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] != res[1][0] and res[0][1] != res[1][1]
    assert res[0][2] == res[1][2] == 2.5


def test_single_process_max_is_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, "cpu") == 3.25
    assert bench.rank_seed(0) == 0
