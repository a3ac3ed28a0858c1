"""Partition of independent propagation jobs over GPUs (one process per GPU).

The jobs of a batch or a serving stream are independent wavepackets: no data
moves between them, so several GPUs share the work by taking disjoint sets of
jobs, with no collective on the data path.  Every rank computes the same
assignment from the same job list (it is deterministic), runs its own jobs on
its own GPU, and only the results (final wavefunctions or observables) travel,
once, to rank 0 over the host process group at the end.

Assignment: every job must fit one GPU's memory on its own (its device
footprint: wavefunction, work copy, potential and operator tables).  Jobs are
taken in decreasing order of estimated cost -- grid points x surfaces x
substeps per step x steps, proportional to the FFT and matvec work -- and each
goes to the rank with the least cost assigned so far among the ranks it fits
(longest-processing-time-first; its makespan is within 4/3 of the optimum).
Ties go to the lower rank, so the result does not depend on anything but the
job list.

    python -m torch.distributed.run --nproc-per-node N -m paper_1903_04946_gb300.partition --jobs 48

serves a seeded stream split this way and prints, on rank 0, the per-rank
shares and the combined throughput.
"""
from __future__ import annotations

import argparse
import json
import time


def job_cost(problem, substeps: int, steps: int) -> float:
    """Work of one job: grid points x surfaces x substeps x steps."""
    return float(problem.points) * problem.S * substeps * steps


def partition(costs, footprints, n_ranks: int, capacity):
    """Longest-processing-time-first assignment of jobs to ranks.

    costs, footprints: per job; capacity: per rank (bytes) or one number.
    Returns (assignment: rank of every job, load: cost per rank).  A job that
    fits no rank raises ValueError."""
    caps = list(capacity) if hasattr(capacity, "__len__") else [capacity] * n_ranks
    if len(caps) != n_ranks:
        raise ValueError("one capacity per rank")
    order = sorted(range(len(costs)), key=lambda j: (-costs[j], j))
    load = [0.0] * n_ranks
    assign = [-1] * len(costs)
    for j in order:
        fits = [r for r in range(n_ranks) if footprints[j] <= caps[r]]
        if not fits:
            raise ValueError(f"job {j} needs {footprints[j]} bytes, more than any rank holds")
        r = min(fits, key=lambda q: (load[q], q))
        assign[j] = r
        load[r] += costs[j]
    return assign, load


def run_partitioned(jobs, runner, costs, footprints, capacity, rank: int, world: int, gather=None):
    """Run this rank's share of `jobs` with `runner(job) -> result` and gather
    {job index: (rank, result)} on rank 0 (None elsewhere).

    `gather(obj)` collects one object per rank on rank 0 (a list, None on the
    other ranks); by default torch.distributed.gather_object over the default
    process group (host objects only: gloo, or NCCL with CPU objects)."""
    assign, load = partition(costs, footprints, world, capacity)
    mine = {}
    for j, r in enumerate(assign):
        if r == rank:
            mine[j] = runner(jobs[j])
    if gather is None:
        import torch.distributed as dist
        out = [None] * world if rank == 0 else None
        dist.gather_object(mine, out, dst=0)
        parts = out
    else:
        parts = gather(mine)
    if rank != 0:
        return None, assign, load
    results = {}
    for r, part in enumerate(parts):
        for j, res in part.items():
            if j in results:
                raise RuntimeError(f"job {j} came back twice")
            results[j] = (r, res)
    return results, assign, load


def main():
    """Serve a seeded job stream split over the ranks of a torchrun launch,
    one GPU per rank (LOCAL_RANK), with the serving loop on each share."""
    import os

    import torch
    import torch.distributed as dist

    from . import serving
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=48)
    ap.add_argument("--seed", type=int, default=1907)
    ap.add_argument("--max-points", type=int, default=1 << 21)
    args = ap.parse_args()
    rank, world = int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist.init_process_group("gloo")  # results and timing only: host objects
    jobs = serving.make_jobs(args.jobs, args.seed, load=1e9, max_points=args.max_points)  # all arrive at once
    costs = [job_cost(j.problem, j.substeps, j.steps_total) for j in jobs]
    foot = [serving.footprint_bytes(j.problem, j.order, j.scheme) for j in jobs]
    cap = int(0.8 * torch.cuda.mem_get_info(local)[0])
    caps = [None] * world
    dist.all_gather_object(caps, cap)
    assign, load = partition(costs, foot, world, caps)
    share = [jobs[j] for j in range(len(jobs)) if assign[j] == rank]
    dist.barrier()
    t0 = time.perf_counter()
    stats = serving.Server(device=local).run(share) if share else {"jobs": 0}
    wall = time.perf_counter() - t0
    obs = {j.jid: [float(x) for x in (j.observables[0], j.observables[1])] for j in share}
    out = [None] * world if rank == 0 else None
    dist.gather_object({"rank": rank, "wall": wall, "stats": stats, "observables": obs}, out, dst=0)
    if rank == 0:
        work = sum(c for c in costs)
        print(json.dumps({"ranks": world, "jobs": len(jobs), "load_per_rank": load,
                          "wall_seconds": max(p["wall"] for p in out),
                          "throughput_amplitude_substeps_per_s": work / max(p["wall"] for p in out),
                          "per_rank": [{k: p[k] for k in ("rank", "wall")} | {"jobs": p["stats"].get("jobs")}
                                       for p in out],
                          "results": sum(len(p["observables"]) for p in out)}))
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
