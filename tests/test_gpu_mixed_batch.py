"""The mixed batch at full size: 512 one-dimensional two-surface packets on
uneven grids (N = 512..8192) and 32 three-dimensional three-surface
instances on mixed 32/64 axes, Suzuki order 6.  Jobs that share a grid form
one batched context (one launch per pass advances all of them); the
contexts run concurrently on their own streams.  Every job keeps its norm;
sampled jobs equal their runs alone bitwise and match the oracle."""
import numpy as np
import pytest

import synth
from gpu_util import assert_parity, gpu_propagate, oracle_propagate, require_gpu

pytestmark = pytest.mark.gpu

DT_1D, DT_3D, STEPS = 1.0, 2000.0 / 128, 2


def test_mixed_batch_full_size():
    dso = require_gpu()
    jobs_1d, jobs_3d = synth.batch_jobs()
    ctxs = []
    for jobs, dt in ((jobs_1d, DT_1D), (jobs_3d, DT_3D)):
        for g in synth.group_batch(jobs):
            ctx = dso.Context(order=6)
            ctx.load_batch([jobs[i] for i in g])
            dso.dso_set_scheme(ctx.ctx, 6, dso.DSO_SUZUKI)
            ctxs.append((ctx, jobs, g, dt))
    # launch every group before reading any result back: the groups overlap
    for ctx, jobs, g, dt in ctxs:
        ctx.propagate(STEPS * dt, dt)
    results = {}
    for ctx, jobs, g, dt in ctxs:
        out = ctx.psi()
        norm, energy, pops = ctx.observables()
        ctx.close()
        assert np.max(np.abs(norm - 1.0)) < 1e-12
        assert np.all(np.isfinite(energy))
        for k, i in enumerate(g):
            results[(id(jobs), i)] = out[k]
    assert len(results) == len(jobs_1d) + len(jobs_3d)
    # sampled jobs: the first of every 1-D grid, one 32^3 and one 64^3 instance
    samples = [(jobs_1d, i, DT_1D) for i in range(len(synth.BATCH_N_1D))] + [(jobs_3d, 0, DT_3D), (jobs_3d, 7, DT_3D)]
    for jobs, i, dt in samples:
        pr = jobs[i]
        got = results[(id(jobs), i)]
        assert np.array_equal(got, gpu_propagate(pr, 6, "suzuki", STEPS * dt, dt)), pr.name
        assert_parity(got, oracle_propagate(pr, 6, "suzuki", STEPS * dt, dt))
