"""The N > 1 bench path on CPU: world-size-2 gloo ranks.

Every rank runs an independent replica (no data-path collective); the job's
figures are the slowest rank's time and the sum of all ranks' units."""
import os
import socket
import sys
from pathlib import Path

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = Path(__file__).resolve().parents[1]


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, str(ROOT))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    elapsed = [0.5, 0.75, 0.25][rank]
    units = [1000, 2500, 7][rank]
    e, u = bench.reduce_over_ranks(dist, elapsed, units, "cpu")
    out[rank] = (e, u, bench.replica_seed(1002, rank), bench._dist())
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_reduce_over_ranks_gloo(world):
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(world, _port(), out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    want_e = max([0.5, 0.75, 0.25][:world])
    want_u = float(sum([1000, 2500, 7][:world]))
    seeds = set()
    for r in range(world):
        e, u, seed, (ws, rank, _local) = res[r]
        assert e == want_e and u == want_u
        assert ws == world and rank == r
        seeds.add(seed)
    assert len(seeds) == world                 # every rank has its own scene


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, str(ROOT))
    import bench
    assert bench.reduce_over_ranks(None, 1.5, 42, "cpu") == (1.5, 42.0)
