"""Failure detection with injected faults, none of which faults the GPU.

* Data corruption of a live state: one job's block of a batched state is
  scaled, or a NaN is written into it, in place through the context's device
  pointer (another kernel writing where it should not).  The norm monitor
  (dso_set_norm_check) must fail the next propagation with DSO_ENUMERIC and
  name that job; after a fresh dso_set_psi the context works again.
* A bounded device wait that gives up: the TMA kernel variant, with the
  diagnostic wait of dso_set_wait_probe on, polls a barrier that no copy ever
  completes; the wait gives up, the next synchronising call returns
  DSO_ETIMEOUT, the propagation itself is unaffected, and the context keeps
  working once the probe is off.
"""
import numpy as np
import pytest

import synth
from gpu_util import assert_parity, oracle_propagate, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dso():
    return require_gpu()


def _batch(dso, B=3):
    jobs = [synth.random_coupled(60 + b, (32, 32), 2, extent=6.0) for b in range(B)]
    for j in jobs[1:]:
        j.mass = jobs[0].mass
    ctx = dso.Context()
    ctx.load_batch(jobs)
    dso.dso_set_scheme(ctx.ctx, 4, dso.DSO_SUZUKI)
    return ctx, jobs


@pytest.mark.parametrize("kind", ["scale", "nan"])
def test_norm_monitor_names_the_corrupted_job(dso, kind):
    import torch
    ctx, jobs = _batch(dso)
    dso.dso_set_norm_check(ctx.ctx, 1e-10)
    ctx.propagate(0.5, 0.25)  # the monitor's reference is taken here; a correct run passes
    view = dso.device_view(dso.dso_psi_device_pointer(ctx.ctx), ctx.shape, np.complex128)
    torch.cuda.synchronize()
    if kind == "scale":
        view[1].mul_(1.001)  # job 1's block
    else:
        view[2, 1, 5, 7] = complex(float("nan"), 0.0)  # one amplitude of job 2
    torch.cuda.synchronize()
    bad = 1 if kind == "scale" else 2
    with pytest.raises(dso.DSOError) as ei:
        ctx.propagate(0.5, 0.25)
    assert ei.value.status == dso.DSO_ENUMERIC
    assert f"job {bad}" in str(ei.value)
    # a fresh state: the context works again and matches the oracle
    ctx.set_psi(np.stack([j.psi0 for j in jobs]))
    ctx.propagate(0.5, 0.25)
    out = ctx.psi()
    ctx.close()
    for b, pr in enumerate(jobs):
        assert_parity(out[b], oracle_propagate(pr, 4, "suzuki", 0.5, 0.25))


def test_unchecked_device_input_caught_by_the_monitor(dso):
    import torch
    pr = synth.random_coupled(3, (16, 16), 2, extent=5.0)
    ctx = dso.Context(pr, order=2)
    dso.dso_set_norm_check(ctx.ctx, 1e-10)
    bad = torch.from_numpy(pr.psi0.copy()).cuda()
    bad[0, 3, 3] = complex(float("inf"), 0.0)
    dso.dso_set_psi(ctx.ctx, bad)  # device input is not checked on the way in
    with pytest.raises(dso.DSOError) as ei:
        ctx.propagate(0.5, 0.25)
    assert ei.value.status == dso.DSO_ENUMERIC and "job 0" in str(ei.value)
    ctx.close()


def test_bounded_wait_gives_up_and_context_recovers(dso, monkeypatch):
    # every pass kind on the TMA variant (lines of 16/32 points, 4 per tile)
    monkeypatch.setenv("DSO_PLAN", "".join(f"{d},{w},2,4,0;" for d in range(3) for w in (0, 1)))
    pr = synth.pyrazine_like(seed=14, n=(16, 32, 16))
    ref = oracle_propagate(pr, 4, "suzuki", 60.0, 30.0)
    ctx = dso.Context(pr, order=4, scheme=dso.DSO_SUZUKI)
    dso.dso_set_wait_probe(ctx.ctx, 1)
    ctx.propagate(60.0, 30.0)
    plan = dso.dso_tuned_plan(ctx.ctx)
    assert all(e.split(",")[2] == "2" for e in plan.strip(";").split(";")), plan
    out = np.empty_like(pr.psi0)
    with pytest.raises(dso.DSOError) as ei:
        dso.dso_get_psi(ctx.ctx, out)
    assert ei.value.status == dso.DSO_ETIMEOUT and "code 5" in str(ei.value)
    assert_parity(out, ref)  # the diagnostic wait left the work unchanged
    # probe off: the same context propagates and reports no error
    dso.dso_set_wait_probe(ctx.ctx, 0)
    ctx.set_psi(pr.psi0)
    ctx.propagate(60.0, 30.0)
    out2 = ctx.psi()
    ctx.close()
    assert np.array_equal(out2, out)
