"""The merged step boundary (dso_set_boundary_merge).

The last a~ action of a time step and the first of the next act on the same
operator back to back (Sec. II F's merge of adjacent actions, across the
step boundary), so they are one action with coefficient a~_last + a~_0.  The
library applies that action from a table of its own by default; the other
form applies the two tables in turn.  Both must match the oracle (which
propagates step by step) within the FP64 parity bound and agree with each
other to round-off, for VTV (merged potential) and TVT (merged kinetic
phase), with the joint and the per-axis kinetic step; and the merged form
must leave no pass with two tables."""
import numpy as np
import pytest

import synth
from gpu_util import assert_parity, oracle_propagate, rel_l2, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dso():
    return require_gpu()


def _run(dso, pr, order, scheme, t, dt, elementary, merged, kinetic):
    el = {"VTV": dso.DSO_VTV, "TVT": dso.DSO_TVT}[elementary]
    ctx = dso.Context(pr, order=order, scheme=dso.SCHEME_CODES[scheme], elementary=el)
    try:
        dso.dso_set_boundary_merge(ctx.ctx, merged)
        dso.dso_set_kinetic_mode(ctx.ctx, kinetic)
        ctx.propagate(t, dt)
        psi = ctx.psi()
        # pass kinds of a middle step: bit 512 a second potential table, 1024 a second kinetic table
        flags = [k["flags"] for k in dso.dso_profile_steps(ctx.ctx, dt, 1)]
        return psi, flags
    finally:
        ctx.close()


@pytest.mark.parametrize("elementary", ["VTV", "TVT"])
@pytest.mark.parametrize("kinetic", ["joint", "axes"])
@pytest.mark.parametrize("order,scheme", [(4, "triple_jump"), (4, "suzuki")])
def test_merged_boundary_matches_two_actions_and_oracle(dso, elementary, kinetic, order, scheme):
    kin = {"joint": dso.DSO_KINETIC_JOINT, "axes": dso.DSO_KINETIC_AXES}[kinetic]
    pr = synth.pyrazine_like(seed=91, n=(32, 32, 16))
    t, dt = 3 * 25.0, 25.0
    merged, fm = _run(dso, pr, order, scheme, t, dt, elementary, 1, kin)
    two, ft = _run(dso, pr, order, scheme, t, dt, elementary, 0, kin)
    assert not any(f & (512 | 1024) for f in fm), fm
    assert any(f & (512 | 1024) for f in ft), ft
    assert rel_l2(merged, two) < 1e-13
    assert_parity(merged, oracle_propagate(pr, order, scheme, t, dt, elementary=elementary))


def test_merged_boundary_one_dimensional_and_first_order(dso):
    """A 1-D grid (the [V F T I] pass) and the first-order TV method, whose
    merged coefficient 1 + 0 is already a unique value."""
    pr = synth.nai_like(seed=92, N=1024)
    a, _ = _run(dso, pr, 6, "suzuki", 4 * 2.0, 2.0, "VTV", 1, dso.DSO_KINETIC_AUTO)
    b, _ = _run(dso, pr, 6, "suzuki", 4 * 2.0, 2.0, "VTV", 0, dso.DSO_KINETIC_AUTO)
    assert rel_l2(a, b) < 1e-13
    assert_parity(a, oracle_propagate(pr, 6, "suzuki", 4 * 2.0, 2.0))
    import paper_1903_04946_gb300 as m
    outs = []
    for merged in (1, 0):
        ctx = m.Context(pr)
        m.dso_set_scheme(ctx.ctx, 1, m.DSO_TRIPLE_JUMP, m.DSO_TV)
        m.dso_set_boundary_merge(ctx.ctx, merged)
        ctx.propagate(3 * 0.5, 0.5)
        outs.append(ctx.psi())
        ctx.close()
    assert rel_l2(outs[0], outs[1]) < 1e-14
    assert_parity(outs[0], oracle_propagate(pr, 1, "triple_jump", 3 * 0.5, 0.5, elementary="TV"))


def test_invalid_merge_value(dso):
    ctx = dso.Context()
    with pytest.raises(dso.DSOError):
        dso.dso_set_boundary_merge(ctx.ctx, 2)
    ctx.close()
