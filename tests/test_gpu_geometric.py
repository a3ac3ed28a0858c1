"""Geometric observables on the device against the oracle (Sec. II A, III A).

* <psi|phi> and omega = -2 Im<psi|phi> from dso_inner agree with the oracle's
  inner product (itself pinned to closed-form Gaussian overlaps), per job.
* The composed split-operator step is unitary, so <U psi|U phi> = <psi|phi>
  and omega is conserved to round-off (App. A).
* The phase at the density maximum (dso_phase_at_density_maximum) matches
  the oracle's on the same propagated state, and its error falls with the
  time step at the order of the method (the phase-convergence study).
"""
import numpy as np
import pytest

import synth
from gpu_util import oracle_propagate, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dso():
    return require_gpu()


def test_inner_matches_oracle(dso):
    from oracle import observables as O
    pr = synth.pyrazine_like(seed=3, n=(32, 16, 32))
    phi = synth.random_state(11, pr)
    ctx = dso.Context(pr, order=2)
    got = ctx.inner(phi)
    import torch
    got_dev = dso.dso_inner(ctx.ctx, torch.from_numpy(phi).cuda())
    ctx.close()
    ref = O.inner(pr, pr.psi0, phi)
    assert abs(got - ref) <= 1e-13 * max(1.0, abs(ref))
    assert got_dev == got


def test_inner_and_omega_conserved_by_propagation(dso):
    from oracle import observables as O
    pr = synth.random_coupled(4, (32, 64), 3, extent=6.0)
    phi0 = synth.random_state(12, pr)
    a = dso.Context(pr, order=6, scheme=dso.DSO_SUZUKI)
    b = dso.Context(pr, order=6, scheme=dso.DSO_SUZUKI)
    b.set_psi(phi0)
    before = a.inner(phi0)
    a.propagate(3.0, 0.5)
    b.propagate(3.0, 0.5)
    phi_t = b.psi()
    after = a.inner(phi_t)
    psi_t = a.psi()
    a.close()
    b.close()
    assert abs(after - before) <= 1e-13
    assert -2 * after.imag == pytest.approx(-2 * before.imag, abs=2e-13)
    # against the oracle's propagation of both states
    ref_psi = oracle_propagate(pr, 6, "suzuki", 3.0, 0.5)
    ref_phi = oracle_propagate(pr, 6, "suzuki", 3.0, 0.5, psi=phi0)
    ref = O.inner(pr, ref_psi, ref_phi)
    assert abs(after - ref) <= 1e-12
    assert O.symplectic_form(pr, ref_psi, ref_phi) == pytest.approx(-2 * after.imag, abs=1e-12)
    assert np.allclose(psi_t, ref_psi, atol=1e-12)


def test_inner_per_job_in_a_batch(dso):
    from oracle import observables as O
    jobs = [synth.random_coupled(20 + b, (16, 32), 2, extent=5.0) for b in range(3)]
    for j in jobs[1:]:
        j.mass = jobs[0].mass
    phis = np.stack([synth.random_state(30 + b, jobs[b]) for b in range(3)])
    ctx = dso.Context()
    ctx.load_batch(jobs)
    got = ctx.inner(phis)
    ctx.close()
    for b in range(3):
        ref = O.inner(jobs[b], jobs[b].psi0, phis[b])
        assert abs(got[b] - ref) <= 1e-13


def test_phase_at_density_maximum_matches_oracle(dso):
    from oracle import observables as O
    pr = synth.nai_like()
    ref = oracle_propagate(pr, 4, "triple_jump", 200.0, 1.0)
    ctx = dso.Context(pr, order=4, scheme=dso.DSO_TRIPLE_JUMP)
    ctx.propagate(200.0, 1.0)
    idx, ph = ctx.phase_at_density_maximum()
    ctx.close()
    ridx, rph = O.phase_at_density_maximum(pr, ref)
    assert list(idx) == list(ridx)
    assert np.abs(np.angle(np.exp(1j * (ph - rph)))).max() < 1e-10


def test_phase_convergence_order(dso):
    from paper_1903_04946_gb300 import phaseconv
    res = phaseconv.study(order=4, scheme="triple_jump", tf=1000.0, ks=(6, 7, 8, 9), ref_k=13)
    assert res["fitted_order"] is not None
    assert res["fitted_order"] == pytest.approx(4.0, abs=0.5), res
    errs = [r["error"] for r in res["rows"]]
    assert all(e1 > e2 for e1, e2 in zip(errs, errs[1:])), res
