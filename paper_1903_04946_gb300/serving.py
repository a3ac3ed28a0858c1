"""Continuous-batching serving loop for propagation jobs.

Requests (a problem, a composition order, a final time and a step) arrive
over time.  The loop keeps every admitted job's wavefunction, potential and
operator tables resident on the device and admits waiting jobs as soon as
their device-memory footprint fits the budget left by the jobs in flight.
Admitted jobs take a slot of one batch (dso_batch_*): each round, one launch
of the batch's work-list kernel advances every slotted job by one composed
step, whatever their grids, schemes and time steps, and jobs join and leave
between rounds.  A job too large for a batch slot (it fills the GPU alone)
advances instead in chunks of time steps on its own CUDA stream, overlapping
with the batch; so does a job above `slot_max_points` points per surface,
whose steps alone keep the GPU busy and would set the length of every round.
With slots=False every job runs that way.
Finished jobs are read back, their latency (finish - arrival) recorded, and
their memory returned to the budget for the next admission.  A job can be
cancelled at any time (`Server.cancel`): a waiting job is dropped, a running
one is retired at its next chunk boundary without a result.  With a log
path, every finished or cancelled job writes one JSON line: its shape, order,
times, latency, and for finished jobs the norm, energy and populations of the
result (FP64 reductions on the device).

All propagation work runs in the library's kernels through the C ABI; this
module only schedules.  Chunking a propagation does not change its result:
a chunk boundary applies the same operations in the same order as the pass
that would have fused them.

    python -m paper_1903_04946_gb300.serving [--jobs 48] [--load 0.8] [--budget-gb 8]

prints one JSON document with p50/p99 latency and throughput.
"""
from __future__ import annotations

import argparse
import json
import time
from dataclasses import dataclass, field

import numpy as np

from . import (DSO_FP64, DSO_TRIPLE_JUMP, Batch, Context, DSOError, dso_busy, dso_scheme_coefficients,
               dso_set_scheme)


@dataclass
class Job:
    jid: int
    problem: object
    order: int
    t: float
    dt: float
    arrival: float = 0.0           # seconds after the start of the run
    scheme: int = DSO_TRIPLE_JUMP
    ctx: object = None
    steps_total: int = 0
    steps_done: int = 0
    admitted: float = -1.0
    finished: float = -1.0
    footprint: int = 0
    cancelled: bool = False
    slot: int = -1                 # batch slot, or -1 (runs alone on its stream)
    result: np.ndarray = field(default=None, repr=False)
    observables: tuple = field(default=None, repr=False)

    @property
    def substeps(self) -> int:
        return len(dso_scheme_coefficients(self.order, self.scheme)[1])


def footprint_bytes(problem, order, scheme=DSO_TRIPLE_JUMP, esz=16) -> int:
    """Device bytes one job holds: psi and the autotuning/observables work
    copy, the FP64 potential, the potential unitaries (one per unique a~, plus
    the merged step-boundary coefficient) and kinetic phases (one per unique
    b~), the twiddles of split axes and small buffers."""
    S, P = problem.S, problem.points
    NP = S * (S + 1) // 2
    a, b, ia, ib, na, nb = dso_scheme_coefficients(order, scheme)
    # four-step twiddles of every axis the library splits (longer than a pass
    # line, or an axis 0 whose S surfaces exceed one tile)
    split = sum(int(x) for d, x in enumerate(problem.n) if x > 4096 or (d == 0 and S * x > 8192))
    return int(2 * S * P * esz + NP * P * 8 + (na + 1) * NP * P * esz + nb * P * esz + split * esz + (1 << 20))


def job_cost_seconds(job, rate=1.2e9) -> float:
    """Rough GPU time of a job at `rate` grid-points x substeps per second
    (per surface triple), used only to pick an arrival rate."""
    return job.problem.points * job.problem.S / 3 * job.substeps * job.steps_total / rate


class Server:
    def __init__(self, device=0, budget_bytes=None, chunk_steps=16, precision=DSO_FP64, slots=True,
                 slot_max_points=1 << 16):
        import torch
        self.device = device
        if budget_bytes is None:
            free, _ = torch.cuda.mem_get_info(device)
            budget_bytes = int(0.8 * free)
        self.budget = budget_bytes
        self.used = 0
        self.peak_used = 0
        self.chunk_steps = chunk_steps
        self.precision = precision
        self._cancel = set()
        self.batch = Batch(device=device, precision=precision) if slots else None
        # a round of the batch lasts as long as its largest job's step: jobs
        # above this many points per surface, which keep the GPU busy alone,
        # run on their own streams instead, so that they do not hold back
        # the small jobs' steps
        self.slot_max_points = slot_max_points
        self.batch_launches = 0

    def cancel(self, jid):
        """Cancel job `jid`: dropped if waiting, retired without a result at
        its next chunk boundary if running."""
        self._cancel.add(jid)

    def _admit(self, job, now):
        job.ctx = Context(device=self.device, precision=self.precision)
        job.ctx.load_problem(job.problem)
        dso_set_scheme(job.ctx.ctx, job.order, job.scheme)
        job.slot = -1
        if self.batch is not None and job.problem.points <= self.slot_max_points:
            try:
                job.slot = self.batch.add(job.ctx, job.t, job.dt)  # the whole run, one step per round
            except DSOError:
                job.slot = -1  # too large for a slot: runs alone on its own stream
        job.admitted = now
        self.used += job.footprint
        self.peak_used = max(self.peak_used, self.used)

    def _retire(self, job, now, keep=True):
        if job.slot >= 0:
            self.batch.retire(job.slot)
            job.slot = -1
        if keep:
            job.result = job.ctx.psi()
            job.observables = job.ctx.observables()
        job.ctx.close()
        job.ctx = None
        job.finished = now
        self.used -= job.footprint

    @staticmethod
    def _log_line(job):
        rec = {"jid": job.jid, "D": job.problem.D, "n": list(job.problem.n), "S": job.problem.S,
               "order": job.order, "steps": job.steps_total, "steps_done": job.steps_done,
               "arrival_s": job.arrival, "admitted_s": job.admitted, "finished_s": job.finished,
               "latency_s": job.finished - job.arrival if job.finished >= 0 else None,
               "cancelled": job.cancelled}
        if job.observables is not None:
            norm, energy, pops = job.observables
            rec.update(norm=float(norm), energy=float(energy), populations=[float(x) for x in pops])
        return json.dumps(rec)

    def run(self, jobs, log=None, on_tick=None):
        """Serve `jobs` (arrival times in seconds from now); returns stats.
        `log`: path of a JSON-lines file, one line per finished or cancelled
        job.  `on_tick(server, now)`: called once per scheduling round."""
        for j in jobs:
            j.steps_total = int(round(j.t / j.dt))
            j.footprint = footprint_bytes(j.problem, j.order, j.scheme, 8 if self.precision else 16)
            if j.footprint > self.budget:
                raise ValueError(f"job {j.jid} needs {j.footprint} bytes, more than the budget")
        waiting = sorted(jobs, key=lambda j: j.arrival)
        active = []
        logf = open(log, "w") if log else None
        t0 = time.perf_counter()
        max_active = 0
        while waiting or active:
            now = time.perf_counter() - t0
            if on_tick is not None:
                on_tick(self, now)
            for job in [j for j in waiting if j.jid in self._cancel]:
                waiting.remove(job)
                job.cancelled = True
                if logf:
                    logf.write(self._log_line(job) + "\n")
            # admit arrived jobs in arrival order while their footprint fits
            while waiting and waiting[0].arrival <= now and self.used + waiting[0].footprint <= self.budget:
                job = waiting.pop(0)
                self._admit(job, now)
                active.append(job)
            max_active = max(max_active, len(active))
            progressed = False
            slotted = [j for j in active if j.slot >= 0]
            if slotted and not self.batch.busy():
                # a round of the batch: retire finished or cancelled slot jobs,
                # then one launch advances every other one by a step
                for job in slotted:
                    job.steps_done = self.batch.status(job.slot)[0]
                    if job.jid in self._cancel or job.steps_done >= job.steps_total:
                        job.cancelled = job.jid in self._cancel and job.steps_done < job.steps_total
                        self._retire(job, time.perf_counter() - t0, keep=not job.cancelled)
                        active.remove(job)
                        if logf:
                            logf.write(self._log_line(job) + "\n")
                if any(j.slot >= 0 for j in active):
                    self.batch.step()
                    self.batch_launches += 1
                progressed = True
            for job in list(active):
                if job.slot >= 0 or dso_busy(job.ctx.ctx):
                    continue
                if job.jid in self._cancel:
                    job.cancelled = True
                    self._retire(job, time.perf_counter() - t0, keep=False)
                    active.remove(job)
                    progressed = True
                    if logf:
                        logf.write(self._log_line(job) + "\n")
                    continue
                if job.steps_done >= job.steps_total:
                    self._retire(job, time.perf_counter() - t0)
                    active.remove(job)
                    progressed = True
                    if logf:
                        logf.write(self._log_line(job) + "\n")
                    continue
                k = min(self.chunk_steps, job.steps_total - job.steps_done)
                job.ctx.propagate(k * job.dt, job.dt)   # asynchronous on the job's stream
                job.steps_done += k
                progressed = True
            if not progressed:
                time.sleep(0.0002)
        wall = time.perf_counter() - t0
        if logf:
            logf.close()
        done = [j for j in jobs if not j.cancelled]
        lat = np.array([j.finished - j.arrival for j in done]) if done else np.zeros(1)
        work = sum(j.problem.points * j.substeps * j.steps_total for j in done)
        return {"jobs": len(jobs), "cancelled": len(jobs) - len(done), "wall_seconds": wall,
                "batch_launches": self.batch_launches,
                "p50_latency_s": float(np.percentile(lat, 50)),
                "p99_latency_s": float(np.percentile(lat, 99)), "mean_latency_s": float(lat.mean()),
                "throughput_grid_pts_substeps_per_s": work / wall, "max_concurrent_jobs": max_active,
                "budget_bytes": self.budget, "peak_footprint_bytes": self.peak_used}


def make_jobs(n_jobs=48, seed=1907, load=0.8, max_points=1 << 21, rate=1.2e9):
    """Seeded Poisson stream of mixed jobs; the arrival rate is set so that the
    offered work is `load` times the GPU's rate."""
    import synth
    jobs = []
    for i in range(n_jobs):
        pr, order, t, dt = synth.serving_job(seed + i, max_points=max_points)
        j = Job(jid=i, problem=pr, order=order, t=t, dt=dt)
        j.steps_total = int(round(t / dt))
        jobs.append(j)
    mean_cost = float(np.mean([job_cost_seconds(j, rate) for j in jobs]))
    lam = load / mean_cost
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / lam, size=n_jobs))
    for j, a in zip(jobs, arrivals):
        j.arrival = float(a)
    return jobs


def run_sequential(jobs, device=0, precision=DSO_FP64):
    """The same jobs one at a time, each alone on the device, in arrival order
    with no waiting for arrivals: the reference for the overlap the serving
    loop gets.  Returns (seconds, grid-pts x substeps per second)."""
    import torch
    work = 0
    t0 = time.perf_counter()
    for j in sorted(jobs, key=lambda j: j.arrival):
        ctx = Context(device=device, precision=precision)
        ctx.load_problem(j.problem)
        dso_set_scheme(ctx.ctx, j.order, j.scheme)
        ctx.propagate(j.t, j.dt)
        torch.cuda.synchronize(device)
        ctx.close()
        work += j.problem.points * j.substeps * int(round(j.t / j.dt))
    secs = time.perf_counter() - t0
    return secs, work / secs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=48)
    ap.add_argument("--load", type=float, default=0.8)
    ap.add_argument("--budget-gb", type=float, default=0.0)
    ap.add_argument("--max-points", type=int, default=1 << 21)
    ap.add_argument("--seed", type=int, default=1907)
    ap.add_argument("--log", default=None, help="JSON-lines file with one record per job")
    ap.add_argument("--no-slots", action="store_true", help="every job on its own stream (no batch slots)")
    ap.add_argument("--sequential", action="store_true",
                    help="also run the same jobs one at a time (no overlap) for comparison")
    args = ap.parse_args()
    jobs = make_jobs(args.jobs, args.seed, args.load, args.max_points)
    srv = Server(budget_bytes=int(args.budget_gb * 2 ** 30) if args.budget_gb else None, slots=not args.no_slots)
    stats = srv.run(jobs, log=args.log)
    stats.update(load=args.load, seed=args.seed, max_points=args.max_points,
                 workload=f"seeded Poisson stream: D in {{1,2,3}}, 2^8..{args.max_points} points per surface, "
                          "S in {2,3,4}, orders 2-8 (triple jump), t in [500, 5000] a.u., complex128")
    if args.sequential:
        secs, rate = run_sequential(make_jobs(args.jobs, args.seed, args.load, args.max_points))
        stats.update(sequential_seconds=secs, sequential_throughput_grid_pts_substeps_per_s=rate)
    print(json.dumps(stats))


if __name__ == "__main__":
    main()
