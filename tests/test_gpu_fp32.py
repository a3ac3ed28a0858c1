"""FP32 storage-and-FFT mode against the FP64 oracle.

In FP32 mode psi, the tables and the FFTs are single precision while the
phase angles, coefficients and reductions stay FP64.  Its error against the
FP64 result is a property of the precision, not a parity bug, so the bound
here is the FP32 one: each FFT adds ~ eps32 * sqrt(log2 P) relative error
(eps32 = 6e-8) and the errors of the n transforms of a run add like a random
walk, so 2e-6 * sqrt(number of FFT passes) bounds the relative L2 error; the
norm (FP64 reduction of FP32 data) drifts by the same order."""
import numpy as np
import pytest

import synth
from gpu_util import gpu_propagate, oracle_propagate, rel_l2, require_gpu

pytestmark = pytest.mark.gpu


def _bound(nfft):
    return 2e-6 * np.sqrt(nfft)


@pytest.mark.parametrize("n,S,order,scheme,nsteps,el", [
    ((64, 64, 64), 3, 4, "triple_jump", 2, "VTV"), ((16, 32, 8), 3, 6, "suzuki", 1, "VTV"),
    ((32, 64), 4, 4, "suzuki", 2, "VTV"), ((1024,), 2, 2, "triple_jump", 20, "VTV"),
    ((4096,), 2, 4, "triple_jump", 2, "VTV"), ((16, 32, 8), 3, 4, "suzuki", 2, "TVT"),
    ((8192,), 2, 4, "suzuki", 2, "VTV")])
def test_fp32_error_vs_fp64_oracle(n, S, order, scheme, nsteps, el):
    require_gpu()
    if len(n) == 3 and S == 3:
        pr = synth.pyrazine_like(seed=21, n=n)
        dt = 2000.0 / 128
    elif n == (1024,):
        pr = synth.nai_like()
        dt = 1.0
    else:
        pr = synth.random_coupled(50 + S, n, S, extent=6.0 if len(n) > 1 else 20.0)
        dt = 0.2
    ref = oracle_propagate(pr, order, scheme, nsteps * dt, dt, elementary=el)
    out = gpu_propagate(pr, order, scheme, nsteps * dt, dt, elementary=el, fp32=True)
    assert out.dtype == np.complex64
    from oracle.coefficients import Splitting
    nsub = Splitting(order, scheme).n_substeps * nsteps
    nfft = 2 * len(n) * nsub
    err = rel_l2(out.astype(np.complex128), ref)
    assert err <= _bound(nfft), (err, _bound(nfft))
    dV = float(np.prod([(pr.qmax[d] - pr.qmin[d]) / pr.n[d] for d in range(pr.D)]))
    norm = np.sqrt(np.sum(np.abs(out.astype(np.complex128)) ** 2) * dV)
    assert abs(norm - 1.0) <= _bound(nfft)


def test_fp32_observables_fp64_reduction():
    dso = require_gpu()
    from oracle import observables as O
    pr = synth.pyrazine_like(seed=22, n=(32, 32, 16))
    ctx = dso.Context(pr, order=4, scheme=dso.DSO_SUZUKI, precision=dso.DSO_FP32)
    ctx.propagate(100.0, 25.0)
    psi = ctx.psi().astype(np.complex128)
    norm, energy, pops = ctx.observables()
    ctx.close()
    # the reductions are FP64 over the FP32 state: they match the oracle's
    # observables of that same state to FP64 accuracy
    assert norm == pytest.approx(O.norm(pr, psi), rel=1e-12)
    assert pops == pytest.approx(O.populations(pr, psi), rel=1e-11, abs=1e-14)
    assert energy == pytest.approx(O.energy(pr, psi), rel=1e-6)  # <T> uses an FP32 FFT of psi


def test_fp32_rejects_fp64_only_variants(monkeypatch):
    require_gpu()
    monkeypatch.setenv("DSO_VARIANT", "2")
    pr = synth.pyrazine_like(seed=23, n=(16, 16, 16))
    ref = oracle_propagate(pr, 2, "triple_jump", 50.0, 25.0)
    out = gpu_propagate(pr, 2, "triple_jump", 50.0, 25.0, fp32=True)   # falls back to the tile kernel
    assert rel_l2(out.astype(np.complex128), ref) < 1e-5


def test_fp32_precision_workload_full_size():
    """The precision workload at its full size (128^3 x 3 surfaces, FP32
    storage and FFTs), one triple-jump order-4 step against the FP64 oracle."""
    require_gpu()
    pr = synth.pyrazine_like(seed=1906, n=(128, 128, 128))
    dt = 2000.0 / 128
    ref = oracle_propagate(pr, 4, "triple_jump", dt, dt)
    out = gpu_propagate(pr, 4, "triple_jump", dt, dt, fp32=True)
    nfft = 2 * 3 * 3
    err = rel_l2(out.astype(np.complex128), ref)
    assert err <= _bound(nfft), (err, _bound(nfft))
