"""The plane pass (dso_set_plane_pass): the kinetic step's passes over the
two last axes of a 3-D grid in one launch.

With a diagonal mass matrix (Eq. (diab_mol_ham)) the kinetic propagator of
Sec. II G factors into one phase per axis, each between its own axis's
forward and inverse FFT (the per-axis form, [F1 T1 I1] [F2 T2 I2]), or is
one phase of the whole grid between full transforms (the joint form, [F1]
[F2 T I2] [I1] on the last two axes).  The plane pass runs either on each
n_1 x n_2 plane of a surface in one cluster of CTAs, with the same FFTs,
tables and products in the same order as the line passes: the result must
be bitwise theirs, for every supported pair of line lengths, both precisions,
both forms, VTV and TVT, merged and unmerged step boundaries (one or two
kinetic tables per pass), batches of jobs and several surface counts; and
within the FP64 parity bound of the oracle."""
import numpy as np
import pytest

import synth
from gpu_util import assert_parity, oracle_propagate, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dso():
    return require_gpu()


def _run(dso, problems, order, scheme, t, dt, plane, elementary="VTV", fp32=False, merged=1, kinetic="axes"):
    el = {"VTV": dso.DSO_VTV, "TVT": dso.DSO_TVT}[elementary]
    ctx = dso.Context(order=order, elementary=el, precision=dso.DSO_FP32 if fp32 else dso.DSO_FP64)
    try:
        if len(problems) == 1:
            ctx.load_problem(problems[0])
        else:
            ctx.load_batch(problems)
        dso.dso_set_scheme(ctx.ctx, order, dso.SCHEME_CODES[scheme], el)
        dso.dso_set_kinetic_mode(ctx.ctx, {"axes": dso.DSO_KINETIC_AXES, "joint": dso.DSO_KINETIC_JOINT}[kinetic])
        dso.dso_set_boundary_merge(ctx.ctx, merged)
        dso.dso_set_plane_pass(ctx.ctx, plane)
        ctx.propagate(t, dt)
        psi = ctx.psi()
        plan = dso.dso_tuned_plan(ctx.ctx)
        # pass kinds of a middle step (bit 32: the plane pass); one more step, after psi was read
        kinds = [(k["axis"], k["flags"], k["launches_per_step"]) for k in dso.dso_profile_steps(ctx.ctx, dt, 1)]
        return psi, kinds, plan
    finally:
        ctx.close()


CASES = [  # grid, surfaces, precision, elementary method, merged step boundary, kinetic form
    ((8, 128, 128), 3, True, "VTV", 1, "axes"),
    ((8, 64, 64), 3, False, "VTV", 1, "axes"),
    ((8, 128, 32), 2, True, "TVT", 0, "axes"),
    ((8, 32, 128), 2, False, "TVT", 1, "axes"),
    ((8, 64, 128), 4, True, "VTV", 0, "axes"),
    ((16, 32, 32), 3, False, "TVT", 0, "axes"),
    ((8, 128, 64), 3, False, "VTV", 1, "axes"),
    ((8, 64, 64), 3, False, "VTV", 1, "joint"),
    ((8, 128, 128), 3, True, "TVT", 0, "joint"),
    ((8, 32, 128), 2, False, "VTV", 0, "joint"),
    ((16, 128, 32), 4, True, "TVT", 1, "joint"),
    ((8, 64, 32), 2, False, "TVT", 1, "joint"),
]


@pytest.mark.parametrize("n,S,fp32,elementary,merged,kinetic", CASES)
def test_plane_pass_bitwise_equals_line_passes(dso, n, S, fp32, elementary, merged, kinetic):
    pr = synth.random_coupled(81 + n[1] + n[2] + S, n, S, extent=6.0)
    t, dt = 3 * 0.3, 0.3
    on, k_on, plan_on = _run(dso, [pr], 4, "suzuki", t, dt, dso.DSO_PLANE_ON, elementary, fp32, merged, kinetic)
    off, k_off, plan_off = _run(dso, [pr], 4, "suzuki", t, dt, dso.DSO_PLANE_OFF, elementary, fp32, merged, kinetic)
    assert np.array_equal(on, off)
    nsub = 5  # Suzuki order 4
    assert any(f & 32 for _, f, _ in k_on) and not any(f & 32 for _, f, _ in k_off)
    # passes per substep: the potential pass and the plane pass, against one
    # pass per axis (per-axis form) or [F1] [F2 T I2] [I1] (joint form)
    assert sum(c for _, _, c in k_on) == 2 * nsub
    assert sum(c for _, _, c in k_off) == (3 if kinetic == "axes" else 4) * nsub
    assert plan_on.endswith("plane;") and "plane" not in plan_off


@pytest.mark.parametrize("kinetic", ["axes", "joint"])
@pytest.mark.parametrize("elementary", ["VTV", "TVT"])
def test_plane_pass_parity(dso, elementary, kinetic):
    pr = synth.pyrazine_like(seed=88, n=(16, 32, 64))
    t, dt = 3 * 25.0, 25.0
    out, _, _ = _run(dso, [pr], 4, "suzuki", t, dt, dso.DSO_PLANE_ON, elementary, kinetic=kinetic)
    assert_parity(out, oracle_propagate(pr, 4, "suzuki", t, dt, elementary=elementary))


@pytest.mark.parametrize("kinetic", ["axes", "joint"])
def test_plane_pass_batch_equals_alone(dso, kinetic):
    base = synth.pyrazine_like(seed=89, n=(8, 64, 64))
    jobs = [base]
    for b in range(1, 3):
        pr = synth.pyrazine_like(seed=89 + b, n=(8, 64, 64))
        pr.mass = base.mass
        jobs.append(pr)
    out, kinds, _ = _run(dso, jobs, 4, "triple_jump", 2 * 30.0, 30.0, dso.DSO_PLANE_ON, kinetic=kinetic)
    assert any(f & 32 for _, f, _ in kinds)
    for b in range(3):
        alone, _, _ = _run(dso, [jobs[b]], 4, "triple_jump", 2 * 30.0, 30.0, dso.DSO_PLANE_OFF, kinetic=kinetic)
        assert np.array_equal(out[b], alone)


def test_plane_auto_gives_the_same_bits(dso):
    """DSO_PLANE_AUTO (the default) picks by timing; either choice must
    give the bits of the line passes."""
    pr = synth.pyrazine_like(seed=92, n=(16, 128, 128))
    auto, _, _ = _run(dso, [pr], 4, "triple_jump", 2 * 15.0, 15.0, dso.DSO_PLANE_AUTO, fp32=True)
    off, _, _ = _run(dso, [pr], 4, "triple_jump", 2 * 15.0, 15.0, dso.DSO_PLANE_OFF, fp32=True)
    assert np.array_equal(auto, off)


def test_plane_pass_not_applied_where_it_does_not_fit(dso):
    """2-D grids and line lengths outside {32, 64, 128}: the mode changes
    nothing."""
    for n, mode in (((64, 64), dso.DSO_KINETIC_JOINT), ((64, 64), dso.DSO_KINETIC_AXES),
                    ((8, 16, 64), dso.DSO_KINETIC_AXES), ((8, 64, 256), dso.DSO_KINETIC_JOINT)):
        pr = synth.random_coupled(93, n, 2, extent=6.0)
        outs = []
        for plane in (dso.DSO_PLANE_ON, dso.DSO_PLANE_OFF):
            ctx = dso.Context(pr, order=4, scheme=dso.DSO_SUZUKI)
            dso.dso_set_kinetic_mode(ctx.ctx, mode)
            dso.dso_set_plane_pass(ctx.ctx, plane)
            ctx.propagate(2 * 0.3, 0.3)
            outs.append(ctx.psi())
            assert not any(k["flags"] & 32 for k in dso.dso_profile_steps(ctx.ctx, 0.3, 1))
            ctx.close()
        assert np.array_equal(outs[0], outs[1])


def test_plane_context_in_a_batch_slot(dso):
    """A context that ran with the plane pass, then advanced in a batch slot
    (line passes only), gives the job's result alone."""
    pr = synth.pyrazine_like(seed=94, n=(8, 32, 64))
    c = dso.Context(pr, order=4, scheme=dso.DSO_SUZUKI)
    dso.dso_set_kinetic_mode(c.ctx, dso.DSO_KINETIC_AXES)
    dso.dso_set_plane_pass(c.ctx, dso.DSO_PLANE_ON)
    c.propagate(0.5, 0.5)
    batch = dso.Batch()
    slot = batch.add(c, 2 * 0.5, 0.5)
    batch.run()
    c = batch.retire(slot)
    out = c.psi()
    c.close()
    batch.close()
    ref = dso.Context(pr, order=4, scheme=dso.DSO_SUZUKI)
    dso.dso_set_kinetic_mode(ref.ctx, dso.DSO_KINETIC_AXES)
    dso.dso_set_plane_pass(ref.ctx, dso.DSO_PLANE_OFF)
    ref.propagate(0.5, 0.5)
    dso.dso_set_pass_limits(ref.ctx, 1024, 2048)
    ref.propagate(2 * 0.5, 0.5)
    want = ref.psi()
    ref.close()
    assert_parity(out, want, tol=1e-13)


def test_invalid_plane_mode(dso):
    ctx = dso.Context()
    with pytest.raises(dso.DSOError):
        dso.dso_set_plane_pass(ctx.ctx, 2)
    ctx.close()
