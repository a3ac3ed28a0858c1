"""Long axes (four-step FFT): parity with the FP64 oracle.

An axis longer than a pass line (4096 points), or an axis 0 whose S surfaces
exceed the potential pass's tile, is transformed as two virtual axes
n = n1 * n2 with twiddles w_n^(k1 i2) between the two FFT passes; the
momentum representation is stored permuted along the split axis, which the
kinetic phases and <T> must follow.  The oracle transforms every axis with its
own radix-2 FFT of the full length, so agreement checks the split, the
twiddles, the permuted kinetic table and the pass ordering at once.
Sizes span the serving workload's range (up to 2^21 points per surface).
"""
import numpy as np
import pytest

import synth
from gpu_util import assert_parity, gpu_propagate, oracle_propagate, rel_l2, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dso():
    return require_gpu()


@pytest.mark.parametrize("N,S,order,scheme,nsteps,extent", [
    (1 << 16, 2, 4, "suzuki", 1, 60.0),      # 256 x 256 virtual axes, Suzuki 4 (5 substeps)
    (1 << 14, 3, 4, "triple_jump", 2, 40.0),  # 128 x 128
    (1 << 13, 4, 6, "triple_jump", 1, 30.0),  # 64 x 128
    (1 << 21, 2, 2, "triple_jump", 2, 400.0),  # 1024 x 2048: the largest serving grid
])
def test_long_1d_parity(dso, N, S, order, scheme, nsteps, extent):
    pr = synth.random_coupled(N % 997 + S, (N,), S, extent=extent)
    dt = 0.25
    ref = oracle_propagate(pr, order, scheme, nsteps * dt, dt)
    out = gpu_propagate(pr, order, scheme, nsteps * dt, dt)
    assert_parity(out, ref)


@pytest.mark.parametrize("n,S", [
    ((8192, 16), 2),       # axis 0 split (64 x 128)
    ((16, 8192), 3),       # last axis split: the kinetic pass runs on its second factor
    ((4096, 8, 8), 3),     # axis 0 split only because S * n0 > 8192
    ((8, 16384, 8), 2),    # a middle axis split
])
def test_multid_split_axis_parity(dso, n, S):
    pr = synth.random_coupled(17 + S, n, S, extent=8.0)
    for el in ("VTV", "TVT"):
        ref = oracle_propagate(pr, 4, "suzuki", 0.4, 0.2, elementary=el)
        out = gpu_propagate(pr, 4, "suzuki", 0.4, 0.2, elementary=el)
        assert_parity(out, ref)


def test_long_axis_observables_and_norm(dso):
    # <T> reads the permuted momentum layout of the split axis
    from oracle import observables as O
    pr = synth.random_coupled(5, (1 << 15,), 2, extent=60.0)
    ctx = dso.Context(pr, order=4, scheme=dso.DSO_SUZUKI)
    ctx.propagate(1.0, 0.25)
    psi = ctx.psi()
    norm, energy, pops = ctx.observables()
    ctx.close()
    assert norm == pytest.approx(O.norm(pr, psi), rel=1e-13)
    assert energy == pytest.approx(O.energy(pr, psi), rel=1e-12)
    assert pops == pytest.approx(O.populations(pr, psi), rel=1e-12, abs=1e-15)
    assert abs(norm - 1.0) < 1e-13


def test_long_axis_time_reversible(dso):
    pr = synth.random_coupled(6, (1 << 17,), 2, extent=100.0)
    ctx = dso.Context(pr, order=6, scheme=dso.DSO_SUZUKI)
    ctx.propagate(2.0, 0.5)
    ctx.propagate(-2.0, -0.5)
    back = ctx.psi()
    ctx.close()
    assert rel_l2(back, pr.psi0) < 1e-12


def test_long_axis_batch_equals_alone(dso):
    jobs = [synth.random_coupled(40 + b, (1 << 14,), 2, extent=40.0) for b in range(3)]
    for j in jobs[1:]:
        j.mass = jobs[0].mass
    ctx = dso.Context()
    ctx.load_batch(jobs)
    dso.dso_set_scheme(ctx.ctx, 4, dso.DSO_TRIPLE_JUMP)
    ctx.propagate(1.0, 0.25)
    batch = ctx.psi()
    ctx.close()
    for b, pr in enumerate(jobs):
        alone = gpu_propagate(pr, 4, "triple_jump", 1.0, 0.25)
        assert np.array_equal(batch[b], alone)


def test_long_axis_fp32(dso):
    pr = synth.random_coupled(8, (1 << 16,), 2, extent=60.0)
    ref = oracle_propagate(pr, 4, "triple_jump", 0.5, 0.25)
    out = gpu_propagate(pr, 4, "triple_jump", 0.5, 0.25, fp32=True)
    # FP32 storage and FFT: error of a few FP32 rounding errors per FFT level
    assert rel_l2(out.astype(np.complex128), ref) < 2e-5


def test_long_axis_variants_are_tile_kernel(dso, monkeypatch):
    # the split axis's first factor runs on the tile kernel only; a plan that
    # asks for another variant there is ignored for that kind, not an error
    pr = synth.random_coupled(9, (1 << 13,), 2, extent=30.0)
    monkeypatch.setenv("DSO_PLAN", "0,1,2,4,0;0,0,1,4,0;1,0,1,4,0;")
    out = gpu_propagate(pr, 4, "suzuki", 0.4, 0.2)
    ref = oracle_propagate(pr, 4, "suzuki", 0.4, 0.2)
    assert_parity(out, ref)
