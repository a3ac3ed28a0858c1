"""User compositions (dso_set_composition): any symmetric set of elementary
coefficients propagates as the oracle's action sequence built from the same
gammas, and the triple-jump gammas reproduce the built-in scheme."""
import numpy as np
import pytest

import synth
from gpu_util import assert_parity, gpu_propagate, oracle_propagate, rel_l2, require_gpu

pytestmark = pytest.mark.gpu


def _custom():
    g = np.array([0.21, -0.13, 0.37, 0.1, 0.37, -0.13, 0.21])
    g[3] = 1.0 - (g.sum() - g[3])
    return g


@pytest.mark.parametrize("el", ["VTV", "TVT"])
def test_custom_composition_parity(el):
    dso = require_gpu()
    from oracle import propagate as P
    pr = synth.pyrazine_like(seed=51, n=(16, 32, 8))
    g = _custom()
    dt = 20.0
    code = dso.DSO_TVT if el == "TVT" else dso.DSO_VTV
    ctx = dso.Context(pr)
    dso.dso_set_composition(ctx.ctx, g, code)
    ctx.propagate(3 * dt, dt)
    out = ctx.psi()
    ctx.close()
    ref = P.propagate(pr, 3 * dt, dt, elementary=el, gammas=g)
    assert_parity(out, ref)


def test_triple_jump_gammas_reproduce_builtin():
    dso = require_gpu()
    pr = synth.pyrazine_like(seed=52, n=(16, 16, 16))
    x = 1.0 / (2.0 - 2.0 ** (1.0 / 3.0))
    ctx = dso.Context(pr)
    dso.dso_set_composition(ctx.ctx, [x, 1.0 - 2.0 * x, x])
    ctx.propagate(100.0, 25.0)
    out = ctx.psi()
    ctx.close()
    assert rel_l2(out, gpu_propagate(pr, 4, "triple_jump", 100.0, 25.0)) < 1e-14
