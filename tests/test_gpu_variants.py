"""Parity of every axis-pass kernel variant against the oracle.  The
autotuner normally picks the fastest; DSO_VARIANT forces one: 0 one CTA per
tile with per-thread loads, 1 persistent CTAs with a tile queue and cp.async
prefetch, 2 TMA bulk tensor copies (lines up to 256 points), 3 persistent
CTAs with TMA copies double-buffered against the FFT work (lines up to 256
points; 1-D grids fall back to another variant), 4 lines of 32..128 points
of the one-surface passes held in registers (the other kinds fall back)."""
import numpy as np
import pytest

import synth
from gpu_util import assert_parity, gpu_propagate, oracle_propagate, require_gpu

pytestmark = pytest.mark.gpu

CASES = [
    ("pyr64", lambda: synth.pyrazine_like(), 4, "triple_jump", 2000.0 / 128, 1),
    ("pyr_mixed", lambda: synth.pyrazine_like(seed=3, n=(16, 32, 8)), 6, "suzuki", 40.0, 1),
    ("rc2d_S4", lambda: synth.random_coupled(2, (32, 64), 4, extent=6.0), 4, "suzuki", 0.3, 2),
    ("rc1d_256", lambda: synth.random_coupled(5, (256,), 2, extent=12.0), 4, "triple_jump", 0.2, 3),
    ("rc1d_S3_128", lambda: synth.random_coupled(6, (128,), 3, extent=10.0), 2, "triple_jump", 0.2, 3),
    ("rc3d_8", lambda: synth.random_coupled(7, (8, 16, 8), 2, extent=4.0), 4, "suzuki", 0.25, 2),
]


@pytest.mark.parametrize("variant", ["0", "1", "2", "3", "4"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_variant_parity(monkeypatch, variant, case):
    require_gpu()
    name, make, order, scheme, dt, nsteps = case
    monkeypatch.setenv("DSO_VARIANT", variant)
    pr = make()
    ref = oracle_propagate(pr, order, scheme, nsteps * dt, dt)
    out = gpu_propagate(pr, order, scheme, nsteps * dt, dt)
    assert_parity(out, ref)


def test_variants_agree_bitwise_or_closely(monkeypatch):
    require_gpu()
    pr = synth.pyrazine_like(seed=8, n=(32, 32, 32))
    outs = []
    for v in ("0", "1", "2", "3", "4"):
        monkeypatch.setenv("DSO_VARIANT", v)
        outs.append(gpu_propagate(pr, 4, "suzuki", 50.0, 25.0))
    for o in outs[1:]:
        # same arithmetic in the same order: the variants differ only in data movement
        assert np.array_equal(o, outs[0])


@pytest.mark.parametrize("variant", ["0", "1", "2", "3", "4"])
@pytest.mark.parametrize("n,S", [((16, 32, 8), 3), ((256,), 2)])
def test_variant_parity_tvt(monkeypatch, variant, n, S):
    require_gpu()
    monkeypatch.setenv("DSO_VARIANT", variant)
    pr = synth.pyrazine_like(seed=4, n=n) if len(n) == 3 else synth.random_coupled(3, n, S, extent=12.0)
    dt = 40.0 if len(n) == 3 else 0.2
    ref = oracle_propagate(pr, 4, "suzuki", 2 * dt, dt, elementary="TVT")
    out = gpu_propagate(pr, 4, "suzuki", 2 * dt, dt, elementary="TVT")
    assert_parity(out, ref)


def test_plan_round_trip(monkeypatch):
    """The configuration the autotuner picks can be written out and forced
    back (DSO_PLAN), giving the same kernels and the same bits."""
    dso = require_gpu()
    pr = synth.pyrazine_like(seed=9, n=(32, 16, 64))
    ctx = dso.Context(pr, order=4, scheme=dso.DSO_SUZUKI)
    ctx.propagate(80.0, 40.0)
    plan = dso.dso_tuned_plan(ctx.ctx)
    a = ctx.psi()
    ctx.close()
    assert plan.count(";") == 6
    # a different configuration, forced: one CTA per tile, small tiles
    monkeypatch.setenv("DSO_PLAN", "0,1,0,1,0;1,0,0,2,0;2,0,0,1,0;")
    c2 = dso.Context(pr, order=4, scheme=dso.DSO_SUZUKI)
    c2.propagate(80.0, 40.0)
    assert dso.dso_tuned_plan(c2.ctx).startswith("0,0,")
    assert "0,1,0,1,0;" in dso.dso_tuned_plan(c2.ctx)
    b = c2.psi()
    c2.close()
    assert np.array_equal(a, b)
    monkeypatch.setenv("DSO_PLAN", plan)
    c3 = dso.Context(pr, order=4, scheme=dso.DSO_SUZUKI)
    c3.propagate(80.0, 40.0)
    assert dso.dso_tuned_plan(c3.ctx) == plan
    assert np.array_equal(a, c3.psi())
    c3.close()


def test_programmatic_dependent_launch_changes_nothing(monkeypatch):
    """Passes launched with programmatic dependent launch (the default) give
    the same bits as plain stream-ordered launches (DSO_PDL=0)."""
    dso = require_gpu()
    pr = synth.pyrazine_like(seed=10, n=(32, 32, 32))
    outs = []
    for flag in ("1", "0"):
        monkeypatch.setenv("DSO_PDL", flag)
        for v in ("0", "2", "3", "4"):
            monkeypatch.setenv("DSO_VARIANT", v)
            outs.append(gpu_propagate(pr, 6, "suzuki", 3 * 25.0, 25.0))
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
