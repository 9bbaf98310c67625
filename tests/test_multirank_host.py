"""The N > 1 path of bench.py on the host: replicas only, so the only
cross-rank step is the aggregation of the timed figures (slowest rank's time,
units summed over ranks).  Two gloo ranks on CPU, rendezvous on 127.0.0.1."""

import os
import socket

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
    ms = [120.0, 150.0][rank]
    units = [1000, 1200][rank]
    out[rank] = bench.aggregate_over_ranks(ms, units, device="cpu")
    ws, r, _ = bench.dist_env()
    assert (ws, r) == (world, rank)
    dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    # every rank sees the whole-job figures: max time, summed units
    assert res[0] == res[1] == (150.0, 2200.0)


def test_aggregate_single_process_is_identity():
    import bench
    assert bench.aggregate_over_ranks(12.5, 40, device="cpu") == (12.5, 40.0)
