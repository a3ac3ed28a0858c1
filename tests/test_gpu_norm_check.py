"""Failure detection by the norm monitor (dso_set_norm_check), with the
failure made on the host: a tolerance tighter than round-off makes an
ordinary, correct propagation report a drift (the detection path), a
realistic tolerance passes, and a batch names the job that drifted."""
import numpy as np
import pytest

import synth
from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def test_norm_check_passes_and_detects():
    dso = require_gpu()
    pr = synth.pyrazine_like(seed=61, n=(16, 16, 16))
    ctx = dso.Context(pr, order=4, scheme=dso.DSO_SUZUKI)
    try:
        dso.dso_set_norm_check(ctx.ctx, 1e-12)
        ctx.propagate(200.0, 25.0)                      # unitary: drift ~1e-15, passes
        dso.dso_set_norm_check(ctx.ctx, 1e-300)         # tighter than round-off
        with pytest.raises(dso.DSOError) as ei:
            ctx.propagate(200.0, 25.0)
        assert ei.value.status == dso.DSO_ENUMERIC
        assert "norm of job 0" in dso.dso_last_error()
        with pytest.raises(dso.DSOError):
            dso.dso_set_norm_check(ctx.ctx, -1.0)
        dso.dso_set_norm_check(ctx.ctx, 0.0)            # off
        ctx.propagate(50.0, 25.0)
    finally:
        ctx.close()


def test_norm_check_uses_each_jobs_own_norm():
    """Jobs of a batch need not be normalised: the reference is each job's
    norm when its state was set."""
    dso = require_gpu()
    jobs = [synth.random_coupled(70 + b, (32, 16), 2, extent=6.0, mass=(1.0, 0.8)) for b in range(3)]
    for b, pr in enumerate(jobs):
        pr.psi0 = pr.psi0 * (1.0 + b)                    # norms 1, 2, 3
    ctx = dso.Context()
    try:
        ctx.load_batch(jobs)
        dso.dso_set_scheme(ctx.ctx, 4, dso.DSO_SUZUKI)
        dso.dso_set_norm_check(ctx.ctx, 1e-12)
        ctx.propagate(0.6, 0.2)
        norm, _, _ = ctx.observables()
        assert np.allclose(norm, [1.0, 2.0, 3.0], rtol=1e-12)
    finally:
        ctx.close()
