"""Partition of independent jobs over GPUs, on CPU.

The assignment (longest processing time first under per-rank memory) is
checked against its guarantees, and the distributed path runs as two gloo
ranks: every rank computes the same assignment, runs its jobs with a stand-in
runner (a host computation on the job's own data, in place of the GPU
propagation), and rank 0 must receive every job's result exactly once, from
the rank the assignment named."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1903_04946_gb300 import partition as PT  # noqa: E402


def test_lpt_balance_and_determinism():
    rng = np.random.default_rng(5)
    costs = list(rng.lognormal(0.0, 1.5, size=200))
    foot = [1] * 200
    for world in (2, 3, 8):
        assign, load = PT.partition(costs, foot, world, 10)
        assert sorted(set(assign)) == list(range(world))
        assert np.allclose(sum(load), sum(costs))
        for r in range(world):
            assert load[r] == pytest.approx(sum(c for c, a in zip(costs, assign) if a == r))
        # LPT makespan bound: max load <= 4/3 OPT, OPT >= max(mean load, largest job)
        lower = max(sum(costs) / world, max(costs))
        assert max(load) <= 4.0 / 3.0 * lower + 1e-9
        assert PT.partition(costs, foot, world, 10) == (assign, load)


def test_memory_capacities_are_respected():
    costs = [5.0, 4.0, 3.0, 3.0, 2.0, 1.0]
    foot = [90, 10, 80, 10, 10, 10]
    assign, load = PT.partition(costs, foot, 3, [100, 50, 50])
    assert assign[0] == 0 and assign[2] == 0  # only rank 0 holds them
    with pytest.raises(ValueError):
        PT.partition([1.0], [200], 2, 100)


def test_job_cost_counts_work():
    import synth
    a = synth.random_coupled(1, (32, 32), 2)
    b = synth.random_coupled(1, (32, 64), 3)
    assert PT.job_cost(b, 25, 10) == pytest.approx(PT.job_cost(a, 25, 10) * 2 * 1.5)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _jobs():
    import synth
    return [synth.random_coupled(100 + i, (8 * (1 + i % 3), 16), 2 + i % 3) for i in range(11)]


def _runner(pr):
    # stands in for the GPU propagation: a result that depends on the job only
    return float(np.sum(np.abs(pr.psi0) ** 2)), pr.name


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    jobs = _jobs()
    costs = [PT.job_cost(p, 5, 3) for p in jobs]
    foot = [p.points * p.S * 16 for p in jobs]
    res, assign, load = PT.run_partitioned(jobs, _runner, costs, foot, 1 << 30, rank, world)
    out[rank] = (res, assign, load)
    dist.destroy_process_group()


def test_two_gloo_ranks_gather_every_result_once():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    res0, assign0, load0 = out[0]
    res1, assign1, load1 = out[1]
    assert res1 is None
    assert assign0 == assign1 and load0 == load1  # the same assignment on every rank
    jobs = _jobs()
    assert sorted(res0) == list(range(len(jobs)))
    for j, (r, val) in res0.items():
        assert r == assign0[j]
        assert val == _runner(jobs[j])
    assert set(assign0) == {0, 1}
