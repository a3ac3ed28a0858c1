"""Batch slots: jobs with uneven grids in one launch per composed step.

Jobs of different dimension, grid, surface count, scheme, order, time step
and number of steps join a batch (dso_batch_add); every dso_batch_step is
one launch of the work-list kernel that advances each unfinished job by one
composed step.  Each job's result must be

* bitwise the result of the same job propagated alone with the batch's pass
  limits (the same arithmetic in the same order), and
* within the parity bound of the FP64 oracle.

Jobs join while others are running (continuous batching) and retired slots
are reused.
"""
import numpy as np
import pytest

import synth
from gpu_util import assert_parity, oracle_propagate, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dso():
    return require_gpu()


# (problem, order, scheme, t, dt, elementary)
def _mixed_jobs():
    jobs = [
        (synth.nai_like(seed=71, N=512), 6, "suzuki", 6.0, 1.0, "VTV"),
        (synth.nai_like(seed=72, N=1024), 4, "triple_jump", 4.0, 2.0, "VTV"),
        (synth.nai_like(seed=73, N=2048), 6, "suzuki", 3.0, 1.0, "VTV"),        # split 32 x 64 in a slot
        (synth.nai_like(seed=74, N=8192), 2, "triple_jump", 5.0, 1.0, "VTV"),   # split 64 x 128
        (synth.pyrazine_like(seed=75, n=(32, 64, 32)), 6, "suzuki", 2 * 2000.0 / 128, 2000.0 / 128, "VTV"),
        (synth.random_coupled(76, (16, 128), 4, extent=6.0), 4, "suzuki", 0.6, 0.2, "TVT"),
        (synth.random_coupled(77, (64,), 3, extent=8.0), 8, "triple_jump", 0.8, 0.2, "VTV"),
        (synth.random_coupled(78, (8, 16, 32), 2, extent=5.0), 2, "triple_jump", 0.0, 0.5, "VTV"),  # no steps
    ]
    return jobs


def _ctx(dso, pr, order, scheme, el, limits=None):
    sch = dso.SCHEME_CODES[scheme]
    elc = {"VTV": dso.DSO_VTV, "TVT": dso.DSO_TVT}[el]
    ctx = dso.Context(pr, order=order, scheme=sch, elementary=elc)
    if limits:
        dso.dso_set_pass_limits(ctx.ctx, *limits)
    return ctx


def test_mixed_batch_equals_alone_and_oracle(dso):
    jobs = _mixed_jobs()
    batch = dso.Batch()
    ctxs, slots = [], []
    for pr, order, scheme, t, dt, el in jobs:
        c = _ctx(dso, pr, order, scheme, el)
        ctxs.append(c)
        slots.append(batch.add(c, t, dt))
    steps = [int(round(t / dt)) for _, _, _, t, dt, _ in jobs]
    while batch.step() > 0:
        pass
    dso.dso_batch_sync(batch.b)
    assert dso.dso_batch_launch_count(batch.b) == max(steps)  # one launch per composed step
    for k, ((pr, order, scheme, t, dt, el), slot) in enumerate(zip(jobs, slots)):
        assert batch.status(slot) == (steps[k], steps[k])
        c = batch.retire(slot)
        out = c.psi()
        c.close()
        alone = _ctx(dso, pr, order, scheme, el, limits=(1024, 2048))
        alone.propagate(t, dt)
        ref_alone = alone.psi()
        alone.close()
        assert np.array_equal(out, ref_alone), k
        if steps[k] == 0:
            assert np.array_equal(out, pr.psi0)
            continue
        assert_parity(out, oracle_propagate(pr, order, scheme, t, dt, elementary=el))
    batch.close()


def test_jobs_join_while_others_run_and_slots_are_reused(dso):
    a = (synth.nai_like(seed=81, N=1024), 4, "triple_jump", 8.0, 1.0, "VTV")
    b = (synth.pyrazine_like(seed=82, n=(16, 32, 16)), 4, "suzuki", 3 * 40.0, 40.0, "VTV")
    c = (synth.random_coupled(83, (32, 32), 3, extent=6.0), 6, "suzuki", 1.0, 0.25, "VTV")
    batch = dso.Batch()
    ca = _ctx(dso, *[a[0], a[1], a[2], a[5]])
    sa = batch.add(ca, a[3], a[4])
    batch.step()
    batch.step()
    cb = _ctx(dso, b[0], b[1], b[2], b[5])
    sb = batch.add(cb, b[3], b[4])  # joins after two of a's steps
    batch.step()
    batch.step()
    batch.step()
    # b finished (3 steps): retire it and put c in its slot
    assert batch.status(sb) == (3, 3)
    out_b = batch.retire(sb).psi()
    cc = _ctx(dso, c[0], c[1], c[2], c[5])
    sc = batch.add(cc, c[3], c[4])
    assert sc == sb
    batch.run()
    out_a = batch.retire(sa).psi()
    out_c = batch.retire(sc).psi()
    for (pr, order, scheme, t, dt, el), out in ((a, out_a), (b, out_b), (c, out_c)):
        al = _ctx(dso, pr, order, scheme, el, limits=(1024, 2048))
        al.propagate(t, dt)
        assert np.array_equal(out, al.psi())
        al.close()
        assert_parity(out, oracle_propagate(pr, order, scheme, t, dt))
    for x in (ca, cb, cc):
        x.close()
    batch.close()


def test_batch_rejects_what_does_not_fit_and_wrong_precision(dso):
    batch = dso.Batch()
    big = synth.random_coupled(90, (1 << 21,), 4, extent=300.0)  # lines above 1024 even after a split
    c = dso.Context(big, order=2)
    with pytest.raises(dso.DSOError):
        batch.add(c, 1.0, 1.0)
    c.propagate(1.0, 1.0)  # still usable alone, with its own limits
    c.close()
    c32 = dso.Context(synth.nai_like(seed=91, N=512), order=2, precision=dso.DSO_FP32)
    with pytest.raises(dso.DSOError):
        batch.add(c32, 1.0, 1.0)
    c32.close()
    batch.close()


def test_fp32_batch_equals_alone(dso):
    jobs = [(synth.nai_like(seed=95, N=4096), 4, "suzuki", 3.0, 1.0, "VTV"),
            (synth.pyrazine_like(seed=96, n=(32, 32, 64)), 4, "triple_jump", 2 * 2000.0 / 128, 2000.0 / 128,
             "VTV")]
    batch = dso.Batch(precision=dso.DSO_FP32)
    slots = []
    for pr, order, scheme, t, dt, el in jobs:
        c = dso.Context(pr, order=order, scheme=dso.DSO_SUZUKI if scheme == "suzuki" else dso.DSO_TRIPLE_JUMP,
                        precision=dso.DSO_FP32)
        slots.append(batch.add(c, t, dt))
    batch.run()
    for (pr, order, scheme, t, dt, el), slot in zip(jobs, slots):
        c = batch.retire(slot)
        out = c.psi()
        c.close()
        al = dso.Context(pr, order=order, scheme=dso.DSO_SUZUKI if scheme == "suzuki" else dso.DSO_TRIPLE_JUMP,
                         precision=dso.DSO_FP32)
        dso.dso_set_pass_limits(al.ctx, 1024, 2048)
        al.propagate(t, dt)
        assert np.array_equal(out, al.psi())
        al.close()
    batch.close()


def test_mixed_batch_config_full_size_one_launch_per_step(dso):
    # the batching configuration: 512 1-D packets on N = 512..8192 and 32 3-D
    # instances on mixed 32/64 axes, Suzuki 6, every job its own slot
    from oracle import observables as O
    jobs_1d, jobs_3d = synth.batch_jobs()
    steps = 2
    batch = dso.Batch()
    held = []
    for jobs, dt in ((jobs_1d, 1.0), (jobs_3d, 2000.0 / 128)):
        for i, pr in enumerate(jobs):
            c = dso.Context(pr, order=6, scheme=dso.DSO_SUZUKI)
            held.append((batch.add(c, steps * dt, dt), pr, dt, i))
    batch.run()
    assert dso.dso_batch_launch_count(batch.b) == steps
    samples = {(id(jobs_1d), i) for i in range(len(synth.BATCH_N_1D))} | {(id(jobs_3d), 0), (id(jobs_3d), 7)}
    for slot, pr, dt, i in held:
        c = batch.retire(slot)
        out = c.psi()
        c.close()
        assert abs(O.norm(pr, out) - 1.0) < 1e-12
        key = (id(jobs_1d) if pr.D == 1 else id(jobs_3d), i)
        if key in samples:
            al = _ctx(dso, pr, 6, "suzuki", "VTV", limits=(1024, 2048))
            al.propagate(steps * dt, dt)
            assert np.array_equal(out, al.psi()), pr.name
            al.close()
            assert_parity(out, oracle_propagate(pr, 6, "suzuki", steps * dt, dt))
    batch.close()


def test_tuning_cache_keeps_pass_limits_apart(dso):
    # the same grid tuned under the batch's limits (a split 64 x 64 axis) and
    # under the defaults (one 4096-point line): each context must use tiles of
    # its own layout
    pr = synth.random_coupled(97, (4096,), 2, extent=20.0)
    for limits in ((1024, 2048), None, (1024, 2048)):
        c = _ctx(dso, pr, 4, "triple_jump", "VTV", limits=limits)
        c.propagate(0.4, 0.2)
        out = c.psi()
        c.close()
        assert_parity(out, oracle_propagate(pr, 4, "triple_jump", 0.4, 0.2))
