"""Batched propagation: B independent jobs on one grid advance together (one
launch per pass for the whole batch).  Every job's result must equal its
result alone (bitwise: the per-line arithmetic does not depend on the
batch), and match the oracle."""
import numpy as np
import pytest

import synth
from gpu_util import assert_parity, gpu_propagate, oracle_propagate, require_gpu

pytestmark = pytest.mark.gpu


def _jobs_3d(B, n=(16, 32, 16)):
    # same grid and masses, different seeded potentials and packets
    return [synth.random_coupled(100 + b, n, 3, extent=6.0, mass=(1.0, 0.7, 1.3)) for b in range(B)]


def _jobs_1d(B, N=512):
    # NaI-like jobs share grid and mass; their potentials and packets differ
    return [synth.nai_like(seed=200 + b, N=N) for b in range(B)]


@pytest.mark.parametrize("el", ["VTV", "TVT"])
def test_batch_3d_equals_alone_and_oracle(el):
    dso = require_gpu()
    jobs = _jobs_3d(5)
    ctx = dso.Context(order=6, scheme=dso.DSO_SUZUKI)
    ctx.load_batch(jobs)
    dso.dso_set_scheme(ctx.ctx, 6, dso.DSO_SUZUKI, dso.DSO_TVT if el == "TVT" else dso.DSO_VTV)
    dt = 0.25
    ctx.propagate(3 * dt, dt)
    out = ctx.psi()
    norm, energy, pops = ctx.observables()
    ctx.close()
    assert out.shape == (5, 3, 16, 32, 16)
    for b, pr in enumerate(jobs):
        alone = gpu_propagate(pr, 6, "suzuki", 3 * dt, dt, elementary=el)
        assert np.array_equal(out[b], alone), b
        assert abs(norm[b] - 1.0) < 1e-12
    for b in (0, 4):
        assert_parity(out[b], oracle_propagate(jobs[b], 6, "suzuki", 3 * dt, dt, elementary=el))
    from oracle import observables as O
    for b in range(5):
        assert energy[b] == pytest.approx(O.energy(jobs[b], out[b]), rel=1e-12)
        assert pops[b] == pytest.approx(O.populations(jobs[b], out[b]), rel=1e-12, abs=1e-15)


def test_batch_1d_many_jobs():
    dso = require_gpu()
    jobs = _jobs_1d(64)
    ctx = dso.Context(order=4)
    ctx.load_batch(jobs)
    dso.dso_set_scheme(ctx.ctx, 4, dso.DSO_TRIPLE_JUMP)
    ctx.propagate(200.0, 1.0)
    out = ctx.psi()
    ctx.close()
    for b in (0, 17, 63):
        alone = gpu_propagate(jobs[b], 4, "triple_jump", 200.0, 1.0)
        assert np.array_equal(out[b], alone)
        assert_parity(out[b], oracle_propagate(jobs[b], 4, "triple_jump", 200.0, 1.0))


@pytest.mark.parametrize("variant", ["0", "1", "2", "3", "4"])
def test_batch_all_variants(monkeypatch, variant):
    dso = require_gpu()
    monkeypatch.setenv("DSO_VARIANT", variant)
    jobs = [synth.random_coupled(300 + b, (32, 16), 3, extent=6.0, mass=(1.0, 0.8)) for b in range(3)]
    ctx = dso.Context(order=4)
    ctx.load_batch(jobs)
    dso.dso_set_scheme(ctx.ctx, 4, dso.DSO_SUZUKI)
    ctx.propagate(0.6, 0.2)
    out = ctx.psi()
    ctx.close()
    for b in range(3):
        assert_parity(out[b], oracle_propagate(jobs[b], 4, "suzuki", 0.6, 0.2))


def test_batch_fp32():
    dso = require_gpu()
    jobs = _jobs_3d(3, n=(32, 32, 32))
    ctx = dso.Context(order=4, precision=dso.DSO_FP32)
    ctx.load_batch(jobs)
    dso.dso_set_scheme(ctx.ctx, 4, dso.DSO_TRIPLE_JUMP)
    ctx.propagate(0.5, 0.25)
    out = ctx.psi()
    ctx.close()
    for b in range(3):
        alone = gpu_propagate(jobs[b], 4, "triple_jump", 0.5, 0.25, fp32=True)
        assert np.array_equal(out[b], alone)


def test_batch_rejects_mismatched_jobs():
    dso = require_gpu()
    ctx = dso.Context()
    with pytest.raises(ValueError):
        ctx.load_batch([synth.pyrazine_like(seed=1, n=(16, 16, 16)), synth.pyrazine_like(seed=2, n=(16, 16, 32))])
    ctx.close()
