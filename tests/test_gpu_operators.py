"""Potential operators precomputed or built per action (dso_set_operator_mode).

Sec. II F trades memory for time: the potential propagators U_a(q) =
exp(-i a dt V(q)) can be stored for every unique coefficient a or built when
an action needs them.  With DSO_OPERATORS_ON_THE_FLY the library stores only
the coefficient-free part of U per grid point (Sec. II H: the closed form's
parameters for S = 2, the eigenvectors and eigenvalues of V for S >= 3) and
assembles each action's table right before its pass with the arithmetic of
the precomputed tables, so the propagation must be bitwise that of the
precomputed tables: for S = 2, 3 (surface 0 decoupled or not) and 4, VTV and
TVT, one or two tables per pass (unmerged step boundaries), FP32, batches of
jobs and every kernel variant; within the FP64 parity bound of the oracle;
with less device memory when the scheme has several unique coefficients."""
import numpy as np
import pytest

import synth
from gpu_util import assert_parity, oracle_propagate, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dso():
    return require_gpu()


def _run(dso, problems, order, scheme, t, dt, mode, elementary="VTV", fp32=False, merged=1):
    el = {"VTV": dso.DSO_VTV, "TVT": dso.DSO_TVT}[elementary]
    ctx = dso.Context(order=order, elementary=el, precision=dso.DSO_FP32 if fp32 else dso.DSO_FP64)
    try:
        if len(problems) == 1:
            ctx.load_problem(problems[0])
        else:
            ctx.load_batch(problems)
        dso.dso_set_scheme(ctx.ctx, order, dso.SCHEME_CODES[scheme], el)
        dso.dso_set_boundary_merge(ctx.ctx, merged)
        dso.dso_set_operator_mode(ctx.ctx, mode)
        ctx.propagate(t, dt)
        return ctx.psi(), dso.dso_operators_on_the_fly(ctx.ctx)
    finally:
        ctx.close()


CASES = [  # problem, order, scheme, elementary, FP32, merged step boundary
    (lambda: synth.pyrazine_like(seed=101, n=(32, 32, 16)), 4, "suzuki", "VTV", False, 1),
    (lambda: synth.pyrazine_like(seed=102, n=(16, 32, 32)), 6, "suzuki", "TVT", False, 0),
    (lambda: synth.random_coupled(103, (32, 64), 2, extent=6.0), 4, "triple_jump", "VTV", False, 0),
    (lambda: synth.random_coupled(104, (16, 16, 32), 3, extent=6.0), 4, "suzuki", "TVT", True, 1),
    (lambda: synth.random_coupled(105, (16, 32, 16), 4, extent=6.0), 4, "triple_jump", "VTV", False, 1),
    (lambda: synth.nai_like(seed=106, N=2048), 6, "optimal", "VTV", True, 0),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_on_the_fly_bitwise_equals_tables(dso, case):
    make, order, scheme, el, fp32, merged = CASES[case]
    pr = make()
    dt = 0.3 if pr.D < 3 or pr.name.startswith("random") else 25.0
    t = 3 * dt
    tab, f_tab = _run(dso, [pr], order, scheme, t, dt, dso.DSO_OPERATORS_TABLES, el, fp32, merged)
    otf, f_otf = _run(dso, [pr], order, scheme, t, dt, dso.DSO_OPERATORS_ON_THE_FLY, el, fp32, merged)
    assert (f_tab, f_otf) == (False, True)
    assert np.array_equal(tab, otf)


def test_on_the_fly_parity(dso):
    pr = synth.pyrazine_like(seed=107, n=(16, 32, 32))
    out, _ = _run(dso, [pr], 6, "suzuki", 3 * 25.0, 25.0, dso.DSO_OPERATORS_ON_THE_FLY)
    assert_parity(out, oracle_propagate(pr, 6, "suzuki", 3 * 25.0, 25.0))


@pytest.mark.parametrize("variant", ["0", "1", "2", "3", "4"])
def test_on_the_fly_every_variant(dso, monkeypatch, variant):
    """Each kernel variant reads the slots (the TMA variants through their
    tensor maps) as it reads the precomputed tables."""
    monkeypatch.setenv("DSO_VARIANT", variant)
    pr = synth.pyrazine_like(seed=108, n=(32, 16, 32))
    tab, _ = _run(dso, [pr], 4, "suzuki", 2 * 25.0, 25.0, dso.DSO_OPERATORS_TABLES, merged=0)
    otf, _ = _run(dso, [pr], 4, "suzuki", 2 * 25.0, 25.0, dso.DSO_OPERATORS_ON_THE_FLY, merged=0)
    assert np.array_equal(tab, otf)


def test_on_the_fly_batch(dso):
    base = synth.pyrazine_like(seed=109, n=(16, 16, 32))
    jobs = [base]
    for b in range(1, 3):
        pr = synth.pyrazine_like(seed=109 + b, n=(16, 16, 32))
        pr.mass = base.mass
        jobs.append(pr)
    tab, _ = _run(dso, jobs, 4, "triple_jump", 2 * 30.0, 30.0, dso.DSO_OPERATORS_TABLES)
    otf, _ = _run(dso, jobs, 4, "triple_jump", 2 * 30.0, 30.0, dso.DSO_OPERATORS_ON_THE_FLY)
    assert np.array_equal(tab, otf)


def test_on_the_fly_uses_less_memory(dso):
    """64^3 x 3 FP64, the optimal order 8 (9 unique potential coefficients,
    each a 25 MB table); built per action, two slots and the per-point
    part."""
    import torch
    pr = synth.pyrazine_like(seed=110, n=(64, 64, 64))
    na = dso.dso_scheme_coefficients(8, dso.DSO_OPTIMAL)[4]
    used = {}
    for mode in (dso.DSO_OPERATORS_TABLES, dso.DSO_OPERATORS_ON_THE_FLY):
        ctx = dso.Context(pr, order=8, scheme=dso.DSO_OPTIMAL)
        dso.dso_set_operator_mode(ctx.ctx, mode)
        ctx.propagate(15.625, 15.625)
        torch.cuda.synchronize()
        free_with = torch.cuda.mem_get_info()[0]
        ctx.close()
        torch.cuda.synchronize()
        used[mode] = torch.cuda.mem_get_info()[0] - free_with
    table = 6 * 16 * 64 ** 3
    assert na >= 6
    # precomputed: na tables; per action: 2 slots and 12 doubles per point (one table's size)
    assert used[dso.DSO_OPERATORS_TABLES] - used[dso.DSO_OPERATORS_ON_THE_FLY] >= (na - 3) * table - (8 << 20)


def test_auto_precomputes_what_fits(dso):
    pr = synth.pyrazine_like(seed=111, n=(16, 16, 16))
    out, fly = _run(dso, [pr], 4, "suzuki", 2 * 25.0, 25.0, dso.DSO_OPERATORS_AUTO)
    assert not fly


def test_batch_slots_take_precomputed_tables(dso):
    pr = synth.pyrazine_like(seed=112, n=(16, 16, 16))
    batch = dso.Batch()
    c = dso.Context(pr, order=4, scheme=dso.DSO_SUZUKI)
    dso.dso_set_operator_mode(c.ctx, dso.DSO_OPERATORS_ON_THE_FLY)
    with pytest.raises(dso.DSOError):
        batch.add(c, 2 * 25.0, 25.0)
    c.close()
    c = dso.Context(pr, order=4, scheme=dso.DSO_SUZUKI)
    c.propagate(25.0, 25.0)  # AUTO
    slot = batch.add(c, 25.0, 25.0)
    batch.run()
    c = batch.retire(slot)
    assert not dso.dso_operators_on_the_fly(c.ctx)
    assert_parity(c.psi(), oracle_propagate(pr, 4, "suzuki", 2 * 25.0, 25.0))
    c.close()
    batch.close()


def test_invalid_operator_mode(dso):
    ctx = dso.Context()
    with pytest.raises(dso.DSOError):
        dso.dso_set_operator_mode(ctx.ctx, 2)
    ctx.close()
