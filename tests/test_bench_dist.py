"""The multi-rank logic of bench.py on CPU: two gloo ranks, each with its own
replica of the benchmarked channel, the timing reduced as the maximum over
ranks and the job's throughput aggregated over ranks (replicas only: nothing
else is exchanged)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench
    from paper_1909_01092_gb300 import workloads as W

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = bench.rank_workload(W, rank)
    ms = 10.0 + 5.0 * rank  # rank 1 is the slower one
    ms_max = bench.max_over_ranks(ms, dist)
    nodes = p["lx"] * p["ly"] * p["lz"]
    out[rank] = (p["replica"], p["seed"], ms_max, bench.aggregate_mlups(nodes, 100, world, ms_max))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    world = 2
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        procs = [mp.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] == 0 and res[1][0] == 1            # distinct replica index: distinct Philox streams
    assert res[0][1] == res[1][1]                       # same seed
    assert res[0][2] == res[1][2] == 15.0               # max over ranks
    nodes = 128 * 128 * 512
    assert res[0][3] == res[1][3] == pytest.approx(nodes * 100 * 2 / 15e-3 / 1e6)
