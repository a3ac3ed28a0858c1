"""First-order VT and TV algorithms (Sec. II E, Eqs. (so_VT), (so_TV)) on the
GPU: parity with the oracle's action sequences, first-order convergence (the
paper's reference against which the composed methods gain), and the
argument checks of dso_set_scheme."""
import numpy as np
import pytest

import synth
from gpu_util import assert_parity, gpu_propagate, oracle_propagate, rel_l2, require_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("el", ["VT", "TV"])
@pytest.mark.parametrize("make,dt,nsteps", [
    (lambda: synth.pyrazine_like(seed=12, n=(16, 32, 8)), 20.0, 3),
    (lambda: synth.random_coupled(13, (256,), 3, extent=12.0), 0.1, 4),
    (lambda: synth.random_coupled(14, (32, 16), 2, extent=6.0), 0.2, 3),
], ids=["pyr3d", "rc1d_S3", "rc2d_S2"])
def test_first_order_parity(el, make, dt, nsteps):
    require_gpu()
    pr = make()
    ref = oracle_propagate(pr, 1, "triple_jump", nsteps * dt, dt, elementary=el)
    out = gpu_propagate(pr, 1, "triple_jump", nsteps * dt, dt, elementary=el)
    assert_parity(out, ref)


def test_vt_and_tv_differ_and_converge_at_first_order():
    """Halving dt halves the error of VT and TV (order 1) but quarters that of
    VTV (order 2); the error is measured against Suzuki order 8 at a small
    step."""
    require_gpu()
    pr = synth.random_coupled(15, (128,), 2, extent=12.0)
    t = 1.6
    ref = gpu_propagate(pr, 8, "suzuki", t, t / 64)
    errs = {}
    for el, order in (("VT", 1), ("TV", 1), ("VTV", 2)):
        e = [rel_l2(gpu_propagate(pr, order, "triple_jump", t, t / n, elementary=el), ref) for n in (32, 64, 128)]
        errs[el] = e
        slope = np.log2(e[1] / e[2])
        assert abs(slope - order) < 0.25, (el, e)
    assert rel_l2(gpu_propagate(pr, 1, "triple_jump", t, t / 32, elementary="VT"),
                  gpu_propagate(pr, 1, "triple_jump", t, t / 32, elementary="TV")) > 1e-6


def test_first_order_argument_checks():
    dso = require_gpu()
    pr = synth.random_coupled(16, (64,), 2, extent=8.0)
    ctx = dso.Context(pr)
    try:
        with pytest.raises(dso.DSOError):
            dso.dso_set_scheme(ctx.ctx, 2, dso.DSO_TRIPLE_JUMP, dso.DSO_VT)   # VT is order 1
        with pytest.raises(dso.DSOError):
            dso.dso_set_scheme(ctx.ctx, 1, dso.DSO_TRIPLE_JUMP, dso.DSO_VTV)  # order 1 needs VT / TV
        dso.dso_set_scheme(ctx.ctx, 1, dso.DSO_SUZUKI, dso.DSO_TV)           # scheme is ignored
        ctx.propagate(0.3, 0.1)
        assert np.all(np.isfinite(ctx.psi()))
    finally:
        ctx.close()
