"""The mixed batch of many wavepackets with uneven grids, three ways.

The workload is the batching configuration: 512 one-dimensional two-surface
NaI-like packets on grids of N = 512..8192 points and 32 three-dimensional
three-surface pyrazine-like instances on mixed 32/64 axes, each with its own
potential and initial state, Suzuki order 6, complex128.  It advances by the
same number of composed steps

* as one batched context per grid shape (jobs that share a grid advance with
  one launch per pass), the contexts on their own streams, all in flight
  together ("contexts");
* as batch slots, one slot per job: every composed step of all 544 jobs is
  one launch of the work-list kernel ("slots, one job each");
* as batch slots, one slot per grid shape, each slot a batched context
  ("slots, one shape each").

Tables are built and the kernels warmed up before timing; the timed region
is the propagation only, synchronised on both sides.  Reported: seconds,
wavepacket-steps per second, grid-point x substeps per second and kernel
launches of each form.

    python -m paper_1903_04946_gb300.mixbatch [--steps 10]

Prints one JSON document.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import (DSO_SUZUKI, Batch, Context, dso_batch_launch_count, dso_batch_sync, dso_launch_count,
               dso_set_scheme)

DT_1D, DT_3D = 1.0, 2000.0 / 128
ORDER = 6
SUBSTEPS = 25  # Suzuki order 6


def _groups(jobs_1d, jobs_3d):
    import synth
    out = []
    for jobs, dt in ((jobs_1d, DT_1D), (jobs_3d, DT_3D)):
        for g in synth.group_batch(jobs):
            out.append(([jobs[i] for i in g], dt))
    return out


def _grouped_context(members):
    ctx = Context(order=ORDER)
    ctx.load_batch(members)
    dso_set_scheme(ctx.ctx, ORDER, DSO_SUZUKI)
    return ctx


def _single_context(pr):
    return Context(pr, order=ORDER, scheme=DSO_SUZUKI)


def run_contexts(groups, steps):
    import torch
    ctxs = [(_grouped_context(m), m, dt) for m, dt in groups]
    for ctx, m, dt in ctxs:  # tables, tuning and the step graph
        ctx.propagate(dt, dt)
        ctx.set_psi(np.stack([p.psi0 for p in m]))
    torch.cuda.synchronize()
    l0 = sum(dso_launch_count(c.ctx) for c, _, _ in ctxs)
    t0 = time.perf_counter()
    for ctx, m, dt in ctxs:
        ctx.propagate(steps * dt, dt)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    launches = sum(dso_launch_count(c.ctx) for c, _, _ in ctxs) - l0
    out = {}
    for ctx, m, dt in ctxs:
        psi = ctx.psi()
        for k, p in enumerate(m):
            out[p.name + str(id(p))] = psi[k]
        ctx.close()
    return secs, launches, out


def run_slots(groups, steps, per_job=True):
    import torch
    # warm-up: one batch of every kind of job for one step (module and kernel load)
    wb = Batch()
    for m, dt in groups:
        c = _single_context(m[0]) if per_job else _grouped_context(m)
        wb.add(c, dt, dt)
    wb.run()
    wb.close()
    batch = Batch()
    held = []
    for m, dt in groups:
        if per_job:
            for p in m:
                c = _single_context(p)
                held.append((batch.add(c, steps * dt, dt), [p]))
        else:
            c = _grouped_context(m)
            held.append((batch.add(c, steps * dt, dt), m))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    batch.run()
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    dso_batch_sync(batch.b)
    launches = dso_batch_launch_count(batch.b)
    out = {}
    for slot, m in held:
        c = batch.retire(slot)
        psi = c.psi()
        for k, p in enumerate(m):
            out[p.name + str(id(p))] = psi if per_job else psi[k]
        c.close()
    batch.close()
    return secs, launches, out


def study(steps=10, seed=1905):
    import synth
    jobs_1d, jobs_3d = synth.batch_jobs(seed)
    groups = _groups(jobs_1d, jobs_3d)
    n_jobs = len(jobs_1d) + len(jobs_3d)
    work = steps * SUBSTEPS * (sum(p.points for p in jobs_1d) + sum(p.points for p in jobs_3d))
    res = {"workload": f"{len(jobs_1d)} 1-D two-surface packets (N = 512..8192) + {len(jobs_3d)} 3-D "
                       f"three-surface instances (32/64 axes), Suzuki order 6, complex128",
           "steps": steps, "jobs": n_jobs, "grid_shapes": len(groups)}
    forms = {}
    base = None
    for name, fn in (("contexts", lambda: run_contexts(groups, steps)),
                     ("slots_one_job_each", lambda: run_slots(groups, steps, True)),
                     ("slots_one_shape_each", lambda: run_slots(groups, steps, False))):
        secs, launches, out = fn()
        forms[name] = {"seconds": secs, "kernel_launches": launches,
                       "per_wavepacket_step_us": secs / (n_jobs * steps) * 1e6,
                       "grid_pts_substeps_per_s": work / secs}
        if base is None:
            base = out
        else:
            # the slot forms use smaller pass lines: round-off level differences only
            diff = max(float(np.sqrt(np.sum(np.abs(out[k] - base[k]) ** 2) / np.sum(np.abs(base[k]) ** 2)))
                       for k in base)
            forms[name]["max_rel_l2_vs_contexts"] = diff
    res["forms"] = forms
    res["slots_vs_contexts"] = forms["contexts"]["seconds"] / forms["slots_one_job_each"]["seconds"]
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=10)
    args = ap.parse_args()
    print(json.dumps(study(args.steps)))


if __name__ == "__main__":
    main()
