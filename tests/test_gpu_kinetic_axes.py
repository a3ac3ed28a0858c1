"""The separable kinetic step (dso_set_kinetic_mode, DSO_KINETIC_AXES).

With a diagonal mass matrix (Eq. (diab_mol_ham)) the kinetic propagator of
Sec. II G is the product over the axes of exp(-i dt p_d^2 / (2 m_d)), whose
factors commute; the library can apply each between its own axis's forward
and inverse FFT, one pass per axis.  The result must match the oracle (which
applies the phase of the whole grid between full transforms) within the
FP64 parity bound, for VTV and TVT, merged step boundaries and graph-replayed
middle steps; the tile and register kernels must agree bit for bit on it;
batches and batch slots must give each job its result alone; and the
default (DSO_KINETIC_AUTO) must take it in FP32 only."""
import numpy as np
import pytest

import synth
from gpu_util import assert_parity, oracle_propagate, rel_l2, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dso():
    return require_gpu()


def _run(dso, problems, order, scheme, t, dt, mode, elementary="VTV", fp32=False, limits=None):
    el = {"VTV": dso.DSO_VTV, "TVT": dso.DSO_TVT}[elementary]
    ctx = dso.Context(order=order, elementary=el, precision=dso.DSO_FP32 if fp32 else dso.DSO_FP64)
    try:
        if len(problems) == 1:
            ctx.load_problem(problems[0])
        else:
            ctx.load_batch(problems)
        dso.dso_set_scheme(ctx.ctx, order, dso.SCHEME_CODES[scheme], el)
        dso.dso_set_kinetic_mode(ctx.ctx, mode)
        # one pass per axis: the plane pass (axes 1 and 2 in one launch) has its own tests
        dso.dso_set_plane_pass(ctx.ctx, dso.DSO_PLANE_OFF)
        if limits:
            dso.dso_set_pass_limits(ctx.ctx, *limits)
        ctx.propagate(t, dt)
        psi = ctx.psi()
        # flags of the pass kinds of a middle step (bit 4: a kinetic phase,
        # bit 16: the phase of one axis); this runs one more step, after psi
        # was read
        kinds = [(k["axis"], k["flags"], k["surfaces"], k["launches_per_step"])
                 for k in dso.dso_profile_steps(ctx.ctx, dt, 1)]
        return psi, kinds
    finally:
        ctx.close()


@pytest.mark.parametrize("elementary", ["VTV", "TVT"])
def test_axes_parity_3d_merged_steps(dso, elementary):
    """Suzuki 4 on a 3-D three-surface model for 3 steps (the first step, a
    graph-replayed middle step with the merged boundary, the final pass)."""
    pr = synth.pyrazine_like(seed=61, n=(32, 32, 32))
    out, kinds = _run(dso, [pr], 4, "suzuki", 3 * 25.0, 25.0, dso.DSO_KINETIC_AXES, elementary)
    assert all(f & 16 for _, f, _, _ in kinds if f & 4), kinds
    assert sum(c for _, _, _, c in kinds) == 3 * 5  # one pass per axis per substep
    assert_parity(out, oracle_propagate(pr, 4, "suzuki", 3 * 25.0, 25.0, elementary=elementary))
    joint, kj = _run(dso, [pr], 4, "suzuki", 3 * 25.0, 25.0, dso.DSO_KINETIC_JOINT, elementary)
    assert not any(f & 16 for _, f, _, _ in kj)
    assert rel_l2(out, joint) < 1e-13


@pytest.mark.parametrize("elementary", ["VTV", "TVT"])
def test_axes_parity_2d_four_surfaces(dso, elementary):
    pr = synth.random_coupled(62, (32, 64), 4, extent=6.0)
    out, _ = _run(dso, [pr], 6, "suzuki", 2 * 0.3, 0.3, dso.DSO_KINETIC_AXES, elementary)
    assert_parity(out, oracle_propagate(pr, 6, "suzuki", 2 * 0.3, 0.3, elementary=elementary))


def test_axes_mixed_lengths_triple_jump(dso):
    pr = synth.pyrazine_like(seed=63, n=(16, 64, 8))
    out, _ = _run(dso, [pr], 8, "triple_jump", 2 * 40.0, 40.0, dso.DSO_KINETIC_AXES)
    assert_parity(out, oracle_propagate(pr, 8, "triple_jump", 2 * 40.0, 40.0))


@pytest.mark.parametrize("fp32", [False, True], ids=["fp64", "fp32"])
def test_axes_tile_and_register_kernels_agree(dso, monkeypatch, fp32):
    pr = synth.pyrazine_like(seed=64, n=(32, 64, 128))
    outs = []
    for v in ("0", "4"):
        monkeypatch.setenv("DSO_VARIANT", v)
        outs.append(_run(dso, [pr], 4, "suzuki", 2 * 25.0, 25.0, dso.DSO_KINETIC_AXES, fp32=fp32)[0])
    assert np.array_equal(outs[0], outs[1])


def test_axes_batch_equals_alone(dso):
    base = synth.pyrazine_like(seed=65, n=(32, 16, 64))
    jobs = [base]
    for b in range(1, 3):
        pr = synth.pyrazine_like(seed=65 + b, n=(32, 16, 64))
        pr.mass = base.mass
        jobs.append(pr)
    out, _ = _run(dso, jobs, 4, "triple_jump", 3 * 30.0, 30.0, dso.DSO_KINETIC_AXES)
    for b in range(3):
        alone, _ = _run(dso, [jobs[b]], 4, "triple_jump", 3 * 30.0, 30.0, dso.DSO_KINETIC_AXES)
        assert np.array_equal(out[b], alone)


def test_axes_batch_slot_equals_alone(dso):
    """A per-axis job in a batch slot, beside a joint one and a 1-D one."""
    specs = [(synth.pyrazine_like(seed=67, n=(32, 64, 32)), dso.DSO_KINETIC_AXES),
             (synth.random_coupled(68, (16, 128), 3, extent=6.0), dso.DSO_KINETIC_JOINT),
             (synth.nai_like(seed=69, N=1024), dso.DSO_KINETIC_AXES)]
    batch = dso.Batch()
    slots = []
    for pr, mode in specs:
        c = dso.Context(pr, order=4, scheme=dso.DSO_SUZUKI)
        dso.dso_set_kinetic_mode(c.ctx, mode)
        slots.append(batch.add(c, 2 * 0.5, 0.5))
    batch.run()
    for (pr, mode), slot in zip(specs, slots):
        c = batch.retire(slot)
        out = c.psi()
        c.close()
        alone, _ = _run(dso, [pr], 4, "suzuki", 2 * 0.5, 0.5, mode, limits=(1024, 2048))
        assert np.array_equal(out, alone)
    batch.close()


def test_default_form_by_precision(dso):
    """Without the call FP64 uses the joint form and FP32 the per-axis one;
    both FP32 forms stay within the FP32 bound of the oracle."""
    pr = synth.pyrazine_like(seed=70, n=(16, 16, 32))
    for fp32 in (False, True):
        ctx = dso.Context(pr, order=2, precision=dso.DSO_FP32 if fp32 else dso.DSO_FP64)
        ctx.propagate(50.0, 50.0)
        kinds = dso.dso_profile_steps(ctx.ctx, 50.0, 1)
        ctx.close()
        if fp32:
            assert all(k["flags"] & 16 for k in kinds if k["flags"] & 4)
        else:
            assert not any(k["flags"] & 16 for k in kinds)
    ref = oracle_propagate(pr, 2, "triple_jump", 2 * 50.0, 50.0)
    for mode in (dso.DSO_KINETIC_AUTO, dso.DSO_KINETIC_JOINT):
        x32, _ = _run(dso, [pr], 2, "triple_jump", 2 * 50.0, 50.0, mode, fp32=True)
        assert rel_l2(x32.astype(np.complex128), ref) < 1e-5


def test_one_axis_and_split_grids_keep_the_joint_form(dso):
    """1-D grids, and grids with an axis split into two virtual axes, have
    no per-axis form: the mode changes nothing."""
    pr = synth.nai_like(seed=71, N=4096)
    a, ka = _run(dso, [pr], 4, "suzuki", 2 * 1.0, 1.0, dso.DSO_KINETIC_AXES)
    b, _ = _run(dso, [pr], 4, "suzuki", 2 * 1.0, 1.0, dso.DSO_KINETIC_JOINT)
    assert not any(f & 16 for _, f, _, _ in ka)
    assert np.array_equal(a, b)
    pr2 = synth.random_coupled(72, (16, 256), 2, extent=6.0)
    a, ka = _run(dso, [pr2], 4, "suzuki", 2 * 0.3, 0.3, dso.DSO_KINETIC_AXES, limits=(64, 2048))  # 256 = 16 x 16
    b, _ = _run(dso, [pr2], 4, "suzuki", 2 * 0.3, 0.3, dso.DSO_KINETIC_JOINT, limits=(64, 2048))
    assert not any(f & 16 for _, f, _, _ in ka)
    assert np.array_equal(a, b)


def test_invalid_mode(dso):
    ctx = dso.Context()
    with pytest.raises(dso.DSOError):
        dso.dso_set_kinetic_mode(ctx.ctx, 2)
    ctx.close()
