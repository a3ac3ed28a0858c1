"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle on
the same seeded inputs, relative L2 <= 1e-12 and every element within
1e-11 of the largest amplitude."""
import numpy as np
import pytest

import synth
from gpu_util import assert_parity, gpu_propagate, oracle_propagate, rel_l2, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dso():
    return require_gpu()


# -- 1-D two-surface NaI-like model at its full size: N = 1024, dt = 1, 2000 steps
@pytest.mark.parametrize("order", [2, 4])
def test_nai_like_full_run(dso, order):
    pr = synth.nai_like()
    ref = oracle_propagate(pr, order, "triple_jump", 2000.0, 1.0)
    out = gpu_propagate(pr, order, "triple_jump", 2000.0, 1.0)
    assert_parity(out, ref)


# -- 3-D three-surface pyrazine-like model at its full size (64^3)
@pytest.mark.parametrize("order,scheme,nsteps", [(2, "triple_jump", 3), (4, "triple_jump", 2), (4, "suzuki", 1)])
def test_pyrazine_like_full_size(dso, order, scheme, nsteps):
    pr = synth.pyrazine_like()
    dt = 2000.0 / 128
    ref = oracle_propagate(pr, order, scheme, nsteps * dt, dt)
    out = gpu_propagate(pr, order, scheme, nsteps * dt, dt)
    assert_parity(out, ref)


# -- every scheme and order on a small mixed-length 3-D grid (tiles of
#    several lines, axes of different lengths)
@pytest.mark.parametrize("scheme", ["triple_jump", "suzuki"])
@pytest.mark.parametrize("order", [2, 4, 6, 8, 10])
def test_all_orders_small_3d(dso, scheme, order):
    pr = synth.pyrazine_like(seed=7, n=(16, 32, 8))
    dt = 40.0
    nsteps = 2 if (scheme == "triple_jump" or order <= 6) else 1
    ref = oracle_propagate(pr, order, scheme, nsteps * dt, dt)
    out = gpu_propagate(pr, order, scheme, nsteps * dt, dt)
    assert_parity(out, ref)


@pytest.mark.parametrize("n,S", [((32, 64), 4), ((64, 8), 2), ((8, 8, 8), 3), ((128, 16), 3)])
def test_2d_3d_random_coupled(dso, n, S):
    pr = synth.random_coupled(21, n, S, extent=6.0)
    ref = oracle_propagate(pr, 6, "suzuki", 0.9, 0.3)
    out = gpu_propagate(pr, 6, "suzuki", 0.9, 0.3)
    assert_parity(out, ref)


@pytest.mark.parametrize("N,S", [(8, 2), (16, 3), (32, 4), (256, 3), (2048, 4), (4096, 2)])
def test_1d_lengths_and_surfaces(dso, N, S):
    pr = synth.random_coupled(N + S, (N,), S, extent=8.0 if N < 64 else 20.0)
    ref = oracle_propagate(pr, 4, "suzuki", 1.2, 0.2)
    out = gpu_propagate(pr, 4, "suzuki", 1.2, 0.2)
    assert_parity(out, ref)


def test_single_step_and_negative_dt(dso):
    pr = synth.random_coupled(3, (32, 16), 2, extent=5.0)
    for t, dt in [(0.4, 0.4), (-1.2, -0.4)]:
        ref = oracle_propagate(pr, 4, "triple_jump", t, dt)
        out = gpu_propagate(pr, 4, "triple_jump", t, dt)
        assert_parity(out, ref)


def test_zero_time_is_identity(dso):
    pr = synth.random_coupled(3, (64,), 3, extent=5.0)
    out = gpu_propagate(pr, 2, "triple_jump", 0.0, 0.5)
    assert np.array_equal(out, pr.psi0)


def test_time_reversible_on_gpu(dso):
    pr = synth.pyrazine_like(seed=9, n=(32, 32, 32))
    ctx = dso.Context(pr, order=6, scheme=dso.DSO_SUZUKI)
    ctx.propagate(200.0, 20.0)
    ctx.propagate(-200.0, -20.0)
    back = ctx.psi()
    ctx.close()
    assert rel_l2(back, pr.psi0) < 1e-12


def test_deterministic(dso):
    pr = synth.pyrazine_like(seed=5, n=(32, 16, 32))
    a = gpu_propagate(pr, 4, "suzuki", 100.0, 25.0)
    b = gpu_propagate(pr, 4, "suzuki", 100.0, 25.0)
    assert np.array_equal(a, b)


def test_observables_match_oracle(dso):
    from oracle import observables as O
    pr = synth.pyrazine_like(seed=4, n=(32, 32, 16))
    ctx = dso.Context(pr, order=4, scheme=dso.DSO_TRIPLE_JUMP)
    ctx.propagate(300.0, 30.0)
    psi = ctx.psi()
    norm, energy, pops = ctx.observables()
    ctx.close()
    assert norm == pytest.approx(O.norm(pr, psi), rel=1e-13)
    assert energy == pytest.approx(O.energy(pr, psi), rel=1e-12)
    assert pops == pytest.approx(O.populations(pr, psi), rel=1e-12, abs=1e-15)
    nai = synth.nai_like()
    ctx = dso.Context(nai, order=2)
    n1, e1, p1 = ctx.observables()
    ctx.close()
    assert e1 == pytest.approx(O.energy(nai, nai.psi0), rel=1e-12)
    assert p1 == pytest.approx(O.populations(nai, nai.psi0), abs=1e-14)


def test_device_buffers_roundtrip(dso):
    import torch
    pr = synth.random_coupled(8, (16, 16), 2, extent=5.0)
    ctx = dso.Context(pr, order=2)
    dev = torch.from_numpy(pr.psi0.copy()).cuda()
    dso.dso_set_psi(ctx.ctx, dev)
    dso.dso_load_potential(ctx.ctx, pr.S, torch.from_numpy(pr.V).cuda())
    dso.dso_set_psi(ctx.ctx, dev)
    ctx.propagate(1.0, 0.25)
    out = torch.empty_like(dev)
    dso.dso_get_psi(ctx.ctx, out)
    torch.cuda.synchronize()
    ctx.close()
    ref = oracle_propagate(pr, 2, "triple_jump", 1.0, 0.25)
    assert_parity(out.cpu().numpy(), ref)


def test_errors_are_reported(dso):
    ctx = dso.dso_create(0)
    try:
        with pytest.raises(dso.DSOError):
            dso.dso_set_grid(ctx, (100,), (0.0,), (1.0,))  # not a power of two
        with pytest.raises(dso.DSOError):
            dso.dso_propagate(ctx, 1.0, 0.1)               # nothing loaded
        pr = synth.random_coupled(1, (32,), 2)
        dso.dso_set_grid(ctx, pr.n, pr.qmin, pr.qmax)
        dso.dso_set_masses(ctx, pr.mass)
        dso.dso_load_potential(ctx, pr.S, pr.V)
        with pytest.raises(dso.DSOError):
            dso.dso_propagate(ctx, 1.0, 0.1)               # psi not set
        dso.dso_set_psi(ctx, pr.psi0)
        with pytest.raises(dso.DSOError):
            dso.dso_propagate(ctx, 1.0, 0.3)               # t/dt not an integer
        with pytest.raises(dso.DSOError):
            dso.dso_set_scheme(ctx, 5)
        bad = pr.psi0.copy()
        bad[0, 3] = np.nan
        with pytest.raises(dso.DSOError) as ei:
            dso.dso_set_psi(ctx, bad)
        assert ei.value.status == dso.DSO_ENUMERIC
        dso.dso_propagate(ctx, 0.0, 0.1)                   # zero steps: a no-op
        with pytest.raises(dso.DSOError):
            dso.dso_set_grid(ctx, (1 << 23,), (0.0,), (1.0,))      # axes up to 2^22 points
        with pytest.raises(dso.DSOError):
            dso.dso_set_grid(ctx, (1 << 16, 1 << 15), (0.0, 0.0), (1.0, 1.0))  # at most 2^30 points
        with pytest.raises(dso.DSOError):
            dso.dso_set_grid(ctx, (4, 64), (0.0, 0.0), (1.0, 1.0))  # axes of at least 8 points
    finally:
        dso.dso_destroy(ctx)


# -- TVT elementary method (Eq. (so_TVT)): kinetic step first and last
@pytest.mark.parametrize("n,S,order,scheme,nsteps", [
    ((64, 64, 64), 3, 4, "triple_jump", 2), ((16, 32, 8), 3, 6, "suzuki", 2), ((32, 64), 2, 4, "suzuki", 3),
    ((1024,), 2, 4, "triple_jump", 3), ((256,), 3, 2, "triple_jump", 1), ((64,), 4, 6, "triple_jump", 2)])
def test_tvt_parity(dso, n, S, order, scheme, nsteps):
    if len(n) == 3 and S == 3:
        pr = synth.pyrazine_like(seed=31, n=n)
        dt = 2000.0 / 128
    else:
        pr = synth.random_coupled(40 + S, n, S, extent=10.0 if len(n) == 1 else 6.0)
        dt = 0.2
    ref = oracle_propagate(pr, order, scheme, nsteps * dt, dt, elementary="TVT")
    out = gpu_propagate(pr, order, scheme, nsteps * dt, dt, elementary="TVT")
    assert_parity(out, ref)


def test_tvt_time_reversible_and_norm(dso):
    pr = synth.random_coupled(9, (32, 32), 2, extent=6.0)
    ctx = dso.Context(pr, order=4, scheme=dso.DSO_SUZUKI, elementary=dso.DSO_TVT)
    ctx.propagate(2.0, 0.25)
    n1, _, _ = ctx.observables()
    ctx.propagate(-2.0, -0.25)
    back = ctx.psi()
    ctx.close()
    assert abs(n1 - 1.0) < 1e-13
    assert rel_l2(back, pr.psi0) < 1e-12


# -- long 1-D grids (S * n > 8192): the axis is split into two virtual axes
@pytest.mark.parametrize("N,S,el", [(8192, 2, "VTV"), (8192, 2, "TVT"), (4096, 3, "VTV"), (4096, 4, "TVT")])
def test_long_1d_grids(dso, N, S, el):
    pr = synth.nai_like(seed=31, N=N) if S == 2 else synth.random_coupled(N + S, (N,), S, extent=40.0)
    dt = 1.0 if S == 2 else 0.2
    ref = oracle_propagate(pr, 4, "suzuki", 3 * dt, dt, elementary=el)
    out = gpu_propagate(pr, 4, "suzuki", 3 * dt, dt, elementary=el)
    assert_parity(out, ref)


# -- the "optimal" non-recursive compositions of orders 6 and 8 (Table II)
@pytest.mark.parametrize("order", [6, 8])
def test_optimal_compositions_parity(dso, order):
    pr = synth.pyrazine_like(seed=41, n=(16, 32, 8))
    ref = oracle_propagate(pr, order, "optimal", 80.0, 40.0)
    out = gpu_propagate(pr, order, "optimal", 80.0, 40.0)
    assert_parity(out, ref)
    nai = synth.nai_like()
    ref = oracle_propagate(nai, order, "optimal", 200.0, 10.0)
    out = gpu_propagate(nai, order, "optimal", 200.0, 10.0)
    assert_parity(out, ref)
