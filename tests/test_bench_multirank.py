"""The multi-GPU bench path on CPU: two gloo ranks, each with its own seeded
wavepacket, combine their timings with a max (the only cross-rank step)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import synth
    seed = bench.rank_seed(rank)
    pr = synth.pyrazine_like(seed=seed, n=(8, 8, 8))
    local_time = 1.0 + rank          # rank 1 is the slower one
    slowest = bench.max_over_ranks(local_time, world)
    value = bench.job_throughput(world, 512, 25, 10, slowest)
    out[rank] = (seed, float(pr.params["omega"][0]), slowest, value)
    dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    (s0, w0, t0, v0), (s1, w1, t1, v1) = out[0], out[1]
    assert s0 != s1 and w0 != w1            # independent inputs per rank
    assert t0 == t1 == 2.0                  # max over ranks
    assert v0 == v1 == pytest.approx(2 * 512 * 25 * 10 / 2.0)
