"""Multi-rank path of bench.py on CPU (gloo, world size 2): each rank processes its own
independent snapshot (no data-path collective); the timing takes the maximum elapsed time over
ranks and the sum of the particles, so the reported value is whole-job throughput."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ws, r, local = bench._dist()
        assert (ws, r, local) == (world, rank, rank)
        bench._barrier(ws)
        # rank r "took" (r + 1) seconds for 1000 (r + 1) particles
        t, u = bench.aggregate(float(rank + 1), 1000.0 * (rank + 1), ws, "cpu")
        seed = bench.synth_seed_for_rank("nfw-2^18-L64", rank)
        out[rank] = (t, u, seed)
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation_and_independent_snapshots():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][:2] == (2.0, 3000.0) and res[1][:2] == (2.0, 3000.0)
    assert res[0][2] != res[1][2]  # each rank draws its own snapshot
