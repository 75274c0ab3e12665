"""The multi-GPU path of bench.py is replicas over disjoint galaxy shards with
no data-path collective: only a barrier and the max-over-ranks time cross
ranks.  Exercised here with world_size 2 on the gloo backend (CPU)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2112_06830_gb300 import synth
    ws, r, _ = bench._dist()
    assert (ws, r) == (world, rank)
    dist.barrier()
    slowest = bench.max_over_ranks(1.5 + rank, dist, "cpu")
    n = 300
    p = synth.make_population(synth.SFH_DPL_QUENCH, n, 1, start=bench.shard_start(rank, n))
    out[rank] = (slowest, p)
    dist.destroy_process_group()


def test_two_rank_replicas_gloo():
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    assert out[0][0] == out[1][0] == 2.5
    from paper_2112_06830_gb300 import synth
    whole = synth.make_population(synth.SFH_DPL_QUENCH, 600, 1)
    np.testing.assert_array_equal(np.concatenate([out[0][1], out[1][1]], axis=1), whole)


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.shard_start(3, 100) == 300
