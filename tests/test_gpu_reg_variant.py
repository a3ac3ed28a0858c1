"""The register-resident axis pass (variant 4) against the tile kernel
(variant 0) and the oracle.

Variant 4 runs passes on lines of 32, 64 and 128 points with each line held
in the registers of 4 or 8 threads and one shared-memory exchange per FFT;
a pass that stages all S surfaces keeps the S lines of a line position in
the same threads, so its potential step is a matvec in registers.  Its
butterflies and matvecs are the tile kernel's -- the same radix plan,
twiddles and inputs in the same order -- so the two give the same bits.  The
grids put every supported length on a strided and on the contiguous axis;
the tuned plan is checked to have used variant 4 for every kind the pass
lists use and the variant takes (VTV: [F_d], [I_d] for d >= 1, the kinetic
pass and [I0 V F0]; TVT also the standalone [F0] and [I0]), so the
comparisons cannot pass on a silent fallback."""
import numpy as np
import pytest

import synth
from gpu_util import assert_parity, oracle_propagate, rel_l2, require_gpu

pytestmark = pytest.mark.gpu

GRIDS = [(32, 64, 128), (128, 64, 32)]


def _run(monkeypatch, variant, problems, order, scheme, t, dt, elementary="VTV", fp32=False):
    import paper_1903_04946_gb300 as dso
    monkeypatch.setenv("DSO_VARIANT", variant)
    el = {"VTV": dso.DSO_VTV, "TVT": dso.DSO_TVT}[elementary]
    ctx = dso.Context(order=order, elementary=el, precision=dso.DSO_FP32 if fp32 else dso.DSO_FP64)
    try:
        if len(problems) == 1:
            ctx.load_problem(problems[0])
        else:
            ctx.load_batch(problems)
        dso.dso_set_scheme(ctx.ctx, order, dso.SCHEME_CODES[scheme], el)
        ctx.propagate(t, dt)
        plan = dso.dso_tuned_plan(ctx.ctx)
        return ctx.psi(), plan
    finally:
        ctx.close()


def _kinds(plan):
    """(axis, 0: one surface staged / 1: all S) -> (variant, tile lines)."""
    out = {}
    for e in plan.strip(";").split(";"):
        d, w, v, g, _ = (int(x) for x in e.split(","))
        out[(d, w)] = (v, g)
    return out


def _check_plan(plan, axes, multi=()):
    """Every one-surface kind on `axes` and every all-surface kind on `multi`
    (those the pass lists use and the variant takes) ran on variant 4."""
    kinds = _kinds(plan)
    for d in axes:
        assert kinds[(d, 0)][0] == 4, plan
    for d in multi:
        assert kinds[(d, 1)][0] == 4, plan


@pytest.mark.parametrize("grid", GRIDS, ids=lambda g: "x".join(map(str, g)))
@pytest.mark.parametrize("fp32", [False, True], ids=["fp64", "fp32"])
def test_reg_variant_bitwise(monkeypatch, grid, fp32):
    require_gpu()
    pr = synth.pyrazine_like(seed=41, n=grid)
    a, _ = _run(monkeypatch, "0", [pr], 4, "suzuki", 2 * 25.0, 25.0, fp32=fp32)
    b, plan = _run(monkeypatch, "4", [pr], 4, "suzuki", 2 * 25.0, 25.0, fp32=fp32)
    # [I0 V F0] stages the 3 surfaces: 128-point lines only in FP32 (registers)
    _check_plan(plan, (1, 2), (0,) if (grid[0] != 128 or fp32) else ())
    assert np.array_equal(a, b)
    if not fp32:
        assert_parity(b, oracle_propagate(pr, 4, "suzuki", 2 * 25.0, 25.0))
    else:
        ref = oracle_propagate(pr, 4, "suzuki", 2 * 25.0, 25.0)
        assert rel_l2(b.astype(np.complex128), ref) < 1e-5


@pytest.mark.parametrize("fp32", [False, True], ids=["fp64", "fp32"])
def test_reg_variant_tvt_two_kinetic_tables(monkeypatch, fp32):
    """TVT: the kinetic pass at a step boundary applies two phase tables."""
    require_gpu()
    pr = synth.pyrazine_like(seed=42, n=(32, 64, 128))
    a, _ = _run(monkeypatch, "0", [pr], 4, "triple_jump", 3 * 20.0, 20.0, elementary="TVT", fp32=fp32)
    b, plan = _run(monkeypatch, "4", [pr], 4, "triple_jump", 3 * 20.0, 20.0, elementary="TVT", fp32=fp32)
    _check_plan(plan, (0, 1, 2), (0,))
    assert np.array_equal(a, b)
    if not fp32:
        assert_parity(b, oracle_propagate(pr, 4, "triple_jump", 3 * 20.0, 20.0, elementary="TVT"))


def test_reg_variant_batch(monkeypatch):
    """A batch of jobs sharing the grid: every job's result equals the tile
    kernel's bit for bit."""
    require_gpu()
    base = synth.pyrazine_like(seed=43, n=(128, 64, 32))
    jobs = [base]
    for b in range(1, 3):
        pr = synth.pyrazine_like(seed=43 + b, n=(128, 64, 32))
        pr.mass = base.mass
        jobs.append(pr)
    a, _ = _run(monkeypatch, "0", jobs, 6, "suzuki", 2 * 30.0, 30.0)
    b, plan = _run(monkeypatch, "4", jobs, 6, "suzuki", 2 * 30.0, 30.0)
    _check_plan(plan, (1, 2))
    assert np.array_equal(a, b)
    assert_parity(b[1], oracle_propagate(jobs[1], 6, "suzuki", 2 * 30.0, 30.0))


def test_reg_variant_two_dimensional(monkeypatch):
    """A 2-D four-surface problem under TVT: a 64-point strided axis (the
    standalone [F0] and the final [I0]) and a 128-point contiguous one."""
    require_gpu()
    pr = synth.random_coupled(44, (64, 128), 4, extent=6.0)
    a, _ = _run(monkeypatch, "0", [pr], 4, "triple_jump", 2 * 0.25, 0.25, elementary="TVT")
    b, plan = _run(monkeypatch, "4", [pr], 4, "triple_jump", 2 * 0.25, 0.25, elementary="TVT")
    _check_plan(plan, (0, 1))
    assert np.array_equal(a, b)
    assert_parity(b, oracle_propagate(pr, 4, "triple_jump", 2 * 0.25, 0.25, elementary="TVT"))


def test_reg_variant_unsupported_kinds_fall_back(monkeypatch):
    """Lines the variant does not take (16 and 8 points; a 32-point axis of
    stride 8, narrower than its tile) keep the tile kernel; the results do
    not change."""
    require_gpu()
    pr = synth.pyrazine_like(seed=45, n=(16, 32, 8))
    a, _ = _run(monkeypatch, "0", [pr], 4, "suzuki", 2 * 40.0, 40.0)
    b, plan = _run(monkeypatch, "4", [pr], 4, "suzuki", 2 * 40.0, 40.0)
    assert all(v != 4 for v, _ in _kinds(plan).values()), plan
    assert np.array_equal(a, b)


@pytest.mark.parametrize("S,grid,fp32", [(2, (32, 64, 64), False), (4, (64, 64, 32), True), (2, (128, 32, 64), True)],
                         ids=["S2_fp64", "S4_fp32", "S2_fp32_128"])
def test_reg_variant_surface_counts(monkeypatch, S, grid, fp32):
    """The passes that stage all S surfaces (the potential step in
    registers) for S = 2 and 4, against the tile kernel bit for bit."""
    require_gpu()
    pr = synth.random_coupled(46 + S, grid, S, extent=5.0)
    a, _ = _run(monkeypatch, "0", [pr], 4, "suzuki", 2 * 0.2, 0.2, fp32=fp32)
    b, plan = _run(monkeypatch, "4", [pr], 4, "suzuki", 2 * 0.2, 0.2, fp32=fp32)
    _check_plan(plan, (1, 2), (0,))
    assert np.array_equal(a, b)
    ref = oracle_propagate(pr, 4, "suzuki", 2 * 0.2, 0.2)
    if fp32:
        assert rel_l2(b.astype(np.complex128), ref) < 1e-5
    else:
        assert_parity(b, ref)


def test_forced_plan_skips_shapes_the_variant_cannot_take(monkeypatch):
    """DSO_PLAN entries naming variant 4 where it does not apply (FP64
    128-point lines of three surfaces: too many amplitudes for a thread's
    registers; a 32-point axis of stride 8, narrower than its tile) are
    ignored: those kinds keep the tile kernel and the propagation runs."""
    dso = require_gpu()
    pr = synth.pyrazine_like(seed=49, n=(128, 32, 8))
    plan = "0,1,4,16,0;1,0,4,32,0;"
    monkeypatch.setenv("DSO_PLAN", plan)
    ctx = dso.Context(pr, order=2)
    ctx.propagate(50.0, 25.0)
    out = ctx.psi()
    kinds = _kinds(dso.dso_tuned_plan(ctx.ctx))
    ctx.close()
    assert kinds[(0, 1)][0] == 0 and kinds[(1, 0)][0] == 0
    monkeypatch.delenv("DSO_PLAN")
    assert_parity(out, oracle_propagate(pr, 2, "triple_jump", 50.0, 25.0))


@pytest.mark.parametrize("fp32", [False, True], ids=["fp64", "fp32"])
def test_reg_variant_split_four_surfaces(monkeypatch, fp32):
    """Four surfaces with surface 0 decoupled: the all-surface pass runs as
    two CTAs per tile (surface 0 with its diagonal entry, surfaces 1-3 with
    their 3 x 3 block); in FP64 that is the only register-resident form the
    32-point lines fit.  Bitwise equal to the tile kernel, within the parity
    bound of the oracle."""
    require_gpu()
    pr = synth.pyrazine_like(seed=50, n=(32, 64, 64), S=4)
    a, _ = _run(monkeypatch, "0", [pr], 4, "suzuki", 2 * 25.0, 25.0, fp32=fp32)
    b, plan = _run(monkeypatch, "4", [pr], 4, "suzuki", 2 * 25.0, 25.0, fp32=fp32)
    _check_plan(plan, (1, 2), (0,))
    assert np.array_equal(a, b)
    ref = oracle_propagate(pr, 4, "suzuki", 2 * 25.0, 25.0)
    if fp32:
        assert rel_l2(b.astype(np.complex128), ref) < 1e-5
    else:
        assert_parity(b, ref)
