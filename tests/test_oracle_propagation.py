"""Pins of the oracle's propagation against closed forms, brute force and the
geometric properties of Sec. II A / Table I:

* free particle (V = 0): the split-operator step is exact for any dt, so it
  must reproduce the analytic spreading Gaussian;
* constant coupling: V commutes with T, so the split-operator step is exact
  and the populations follow the Rabi formula;
* uncoupled harmonic surfaces: coherent states have a closed form; the
  composed methods converge to it at order n;
* tiny grids: dense exp(-iHt) is the dt -> 0 limit of every method;
* unitarity/symplecticity, time reversibility (and its failure for VT),
  pruned == unpruned, energy error of order n.
"""
import numpy as np
import pytest

import synth
from oracle import brute, observables as O, propagate as P
from oracle.coefficients import OPTIMAL, SUZUKI, TRIPLE_JUMP


def _problem_1d(V, psi0, n, qmin, qmax, mass):
    S = psi0.shape[0]
    return synth.Problem(n=(n,), qmin=(qmin,), qmax=(qmax,), mass=(mass,), S=S,
                         V=np.asarray(V, float), psi0=np.asarray(psi0, complex))


def _free_gaussian(q, t, q0, p0, sigma, m):
    tau = t / (m * sigma ** 2)
    return ((np.pi * sigma ** 2) ** -0.25 / np.sqrt(1 + 1j * tau)
            * np.exp(-(q - q0 - p0 * t / m) ** 2 / (2 * sigma ** 2 * (1 + 1j * tau))
                     + 1j * p0 * (q - q0) - 1j * p0 ** 2 * t / (2 * m)))


@pytest.mark.parametrize("elementary,order,scheme,dt", [
    (P.VTV, 2, TRIPLE_JUMP, 0.5), (P.VTV, 4, SUZUKI, 0.25), (P.TVT, 2, TRIPLE_JUMP, 1.0),
    (P.VT, 2, TRIPLE_JUMP, 0.4)])
def test_free_particle_exact(elementary, order, scheme, dt):
    n, qmin, qmax, m = 256, -20.0, 20.0, 1.3
    q = np.linspace(qmin, qmax, n, endpoint=False)
    q0, p0, sigma, t = -1.0, 1.2, 1.0, 2.0
    psi0 = np.stack([_free_gaussian(q, 0.0, q0, p0, sigma, m),
                     0.5j * _free_gaussian(q, 0.0, q0, p0, sigma, m)])
    pr = _problem_1d(np.zeros((3, n)), psi0, n, qmin, qmax, m)
    out = P.propagate(pr, t, dt, order=order, scheme=scheme, elementary=elementary)
    ref = np.stack([_free_gaussian(q, t, q0, p0, sigma, m),
                    0.5j * _free_gaussian(q, t, q0, p0, sigma, m)])
    assert O.rel_l2(out, ref) < 1e-12


@pytest.mark.parametrize("order,scheme,elementary", [
    (2, TRIPLE_JUMP, P.VTV), (4, TRIPLE_JUMP, P.VTV), (6, SUZUKI, P.VTV), (4, SUZUKI, P.TVT)])
def test_constant_coupling_rabi_exact(order, scheme, elementary):
    n, qmin, qmax, m = 64, -8.0, 8.0, 1.0
    eps, c, v0 = 0.03, 0.11, -0.2
    V = np.zeros((3, n))
    V[0] = v0 + eps
    V[1] = c
    V[2] = v0 - eps
    psi0 = np.zeros((2, n), complex)
    psi0[0] = synth.gaussian((n,), (qmin,), (qmax,), (0.5,), (0.3,), (1.0,))
    pr = _problem_1d(V, psi0, n, qmin, qmax, m)
    Om = np.hypot(eps, c)
    for t, dt in [(3.7, 0.37), (11.1, 3.7)]:
        out = P.propagate(pr, t, dt, order=order, scheme=scheme, elementary=elementary)
        pops = O.populations(pr, out)
        assert pops[1] == pytest.approx(c ** 2 / Om ** 2 * np.sin(Om * t) ** 2, abs=1e-13)
        assert pops.sum() == pytest.approx(1.0, abs=1e-13)
        # the spatial part moves freely and the surface amplitudes are the 2x2 propagator's
        ph = np.exp(-1j * v0 * t)
        a00 = ph * (np.cos(Om * t) - 1j * eps / Om * np.sin(Om * t))
        a10 = ph * (-1j * c / Om * np.sin(Om * t))
        free = P.propagate(_problem_1d(np.zeros((3, n)), psi0, n, qmin, qmax, m), t, dt)
        assert O.rel_l2(out, np.stack([a00 * free[0], a10 * free[0]])) < 1e-12


def _coherent(x, xbar, pbar, m, w):
    """(m w/pi)^{1/4} exp(-(m w/2)(x - xbar)^2 + i pbar x - i xbar pbar / 2)."""
    return ((m * w / np.pi) ** 0.25
            * np.exp(-0.5 * m * w * (x - xbar) ** 2 + 1j * pbar * x - 0.5j * xbar * pbar))


def _harmonic_case():
    n, qmin, qmax, m, w = 128, -12.0, 12.0, 1.0, 1.0
    q = np.linspace(qmin, qmax, n, endpoint=False)
    centres, E = (-1.0, 1.0), (0.0, 0.5)
    x0, p0 = 2.0, 0.5
    V = np.zeros((3, n))
    V[0] = 0.5 * m * w ** 2 * (q - centres[0]) ** 2 + E[0]
    V[2] = 0.5 * m * w ** 2 * (q - centres[1]) ** 2 + E[1]
    psi0 = np.stack([_coherent(q - centres[s], x0, p0, m, w) for s in range(2)]) / np.sqrt(2)
    pr = _problem_1d(V, psi0, n, qmin, qmax, m)

    def exact(t):
        xb = x0 * np.cos(w * t) + p0 / (m * w) * np.sin(w * t)
        pb = p0 * np.cos(w * t) - m * w * x0 * np.sin(w * t)
        return np.stack([np.exp(-1j * (E[s] + 0.5 * w) * t) * _coherent(q - centres[s], xb, pb, m, w)
                         for s in range(2)]) / np.sqrt(2)
    return pr, exact


@pytest.mark.parametrize("order,scheme,elementary,dts", [
    (2, TRIPLE_JUMP, P.VTV, (0.05, 0.025)),
    (2, TRIPLE_JUMP, P.TVT, (0.05, 0.025)),
    (4, TRIPLE_JUMP, P.VTV, (0.2, 0.1)),
    (4, SUZUKI, P.VTV, (0.4, 0.2)),
    (6, TRIPLE_JUMP, P.VTV, (0.4, 0.2)),
    (6, OPTIMAL, P.VTV, (0.4, 0.2)),
    (8, OPTIMAL, P.VTV, (1.0, 0.5)),
])
def test_harmonic_coherent_state_convergence_order(order, scheme, elementary, dts):
    pr, exact = _harmonic_case()
    t = 2.0
    ref = exact(t)
    errs = [O.l2_error(pr, P.propagate(pr, t, dt, order, scheme, elementary), ref) for dt in dts]
    slope = np.log2(errs[0] / errs[1])
    assert abs(slope - order) < 0.3, (errs, slope)
    assert errs[1] < 1e-3


def test_harmonic_coherent_state_high_order_accuracy():
    pr, exact = _harmonic_case()
    out = P.propagate(pr, 2.0, 0.05, order=8, scheme=SUZUKI)
    assert O.l2_error(pr, out, exact(2.0)) < 1e-10


def _tiny():
    return synth.random_coupled(11, (16,), 2, extent=4.0, mass=(1.0,), coupling=0.3)


@pytest.mark.parametrize("order,scheme,elementary", [
    (2, TRIPLE_JUMP, P.VTV), (2, TRIPLE_JUMP, P.TVT), (4, TRIPLE_JUMP, P.VTV),
    (4, SUZUKI, P.VTV), (6, SUZUKI, P.VTV)])
def test_brute_force_limit_and_order(order, scheme, elementary):
    pr = _tiny()
    t = 1.0
    ref = brute.exact_propagate(pr, pr.psi0, t)
    dts = (1 / 8, 1 / 16)
    errs = [O.l2_error(pr, P.propagate(pr, t, dt, order, scheme, elementary), ref) for dt in dts]
    slope = np.log2(errs[0] / errs[1])
    assert abs(slope - order) < 0.35, (errs, slope)
    fine = P.propagate(pr, t, 1 / 64, 8, SUZUKI, elementary)
    assert O.l2_error(pr, fine, ref) < 1e-11


@pytest.mark.parametrize("order,dts", [(6, (0.1, 0.05)), (8, (0.125, 0.0625))])
def test_optimal_compositions_order_on_an_anharmonic_problem(order, dts):
    """The tabulated optimal compositions reach their order on a coupled,
    anharmonic grid problem, where every order condition counts (on a
    quadratic Hamiltonian some of them coincide), against dense exp(-iHt)."""
    pr = _tiny()
    t = 1.0
    ref = brute.exact_propagate(pr, pr.psi0, t)
    errs = [O.l2_error(pr, P.propagate(pr, t, dt, order, OPTIMAL), ref) for dt in dts]
    slope = np.log2(errs[0] / errs[1])
    assert abs(slope - order) < 0.35, (errs, slope)


def test_brute_force_2d_three_surfaces():
    pr = synth.random_coupled(5, (4, 8), 3, extent=3.0, mass=(1.0, 0.7), coupling=0.2)
    ref = brute.exact_propagate(pr, pr.psi0, 0.5)
    out = P.propagate(pr, 0.5, 0.5 / 16, 8, SUZUKI)
    assert O.l2_error(pr, out, ref) < 1e-11


@pytest.mark.parametrize("order,scheme", [(2, TRIPLE_JUMP), (4, SUZUKI), (6, TRIPLE_JUMP)])
def test_norm_inner_product_symplectic_conserved(order, scheme):
    pr = synth.random_coupled(3, (64,), 2, extent=8.0)
    phi = synth.random_state(4, pr)
    prop = P.Propagator(pr)
    seq = P.action_sequence(P.VTV, order, scheme)
    a = prop.run(pr.psi0, seq, 0.3, 40)
    b = prop.run(phi, seq, 0.3, 40)
    assert O.norm(pr, a) == pytest.approx(O.norm(pr, pr.psi0), abs=1e-13)
    assert abs(O.inner(pr, a, b) - O.inner(pr, pr.psi0, phi)) < 1e-13
    assert O.symplectic_form(pr, a, b) == pytest.approx(O.symplectic_form(pr, pr.psi0, phi), abs=1e-13)


@pytest.mark.parametrize("elementary,order,scheme", [
    (P.VTV, 2, TRIPLE_JUMP), (P.TVT, 2, TRIPLE_JUMP), (P.VTV, 4, TRIPLE_JUMP), (P.VTV, 6, SUZUKI)])
def test_time_reversible(elementary, order, scheme):
    pr = synth.random_coupled(8, (64,), 2, extent=8.0, coupling=0.05)
    prop = P.Propagator(pr)
    seq = P.action_sequence(elementary, order, scheme)
    fwd = prop.run(pr.psi0, seq, 0.4, 25)
    back = prop.run(fwd, seq, -0.4, 25)
    assert O.l2_error(pr, back, pr.psi0) < 1e-12


def test_first_order_not_time_reversible():
    """Negative control (Table I, Fig. geom_prop (d)): VT forward then
    backward does not return psi0."""
    pr = synth.random_coupled(8, (64,), 2, extent=8.0, coupling=0.05)
    prop = P.Propagator(pr)
    seq = P.action_sequence(P.VT)
    back = prop.run(prop.run(pr.psi0, seq, 0.4, 25), seq, -0.4, 25)
    assert O.l2_error(pr, back, pr.psi0) > 1e-3


@pytest.mark.parametrize("order,scheme", [(4, TRIPLE_JUMP), (4, SUZUKI), (6, SUZUKI)])
def test_pruned_equals_unpruned(order, scheme):
    pr = synth.random_coupled(2, (32,), 2, extent=6.0)
    a = P.propagate(pr, 3.0, 0.5, order, scheme, pruned=True)
    b = P.propagate(pr, 3.0, 0.5, order, scheme, pruned=False)
    assert O.rel_l2(a, b) < 1e-13


def test_dft_and_fft_paths_agree():
    pr = synth.random_coupled(4, (16, 8), 2, extent=4.0)
    seq = P.action_sequence(P.VTV, 4, SUZUKI)
    a = P.Propagator(pr).run(pr.psi0, seq, 0.2, 5)
    b = P.Propagator(pr, dft=True).run(pr.psi0, seq, 0.2, 5)
    assert O.rel_l2(a, b) < 1e-13


@pytest.mark.parametrize("order,scheme,dts", [(2, TRIPLE_JUMP, (0.1, 0.05)), (4, SUZUKI, (0.4, 0.2))])
def test_energy_error_order(order, scheme, dts):
    pr = synth.random_coupled(6, (64,), 2, extent=8.0, coupling=0.1)
    E0 = O.energy(pr, pr.psi0)
    t = 2.0
    errs = [abs(O.energy(pr, P.propagate(pr, t, dt, order, scheme)) - E0) for dt in dts]
    slope = np.log2(errs[0] / errs[1])
    assert abs(slope - order) < 0.4, (errs, slope)


def test_observables_closed_forms():
    n, qmin, qmax, m, k = 256, -15.0, 15.0, 1.7, 0.6
    q = np.linspace(qmin, qmax, n, endpoint=False)
    q0, p0, sigma = 0.7, -1.1, 1.3
    V = np.zeros((3, n))
    V[0] = 0.5 * k * q ** 2
    V[2] = 0.5 * k * q ** 2 + 0.25
    psi0 = np.stack([synth.gaussian((n,), (qmin,), (qmax,), (q0,), (p0,), (sigma,)) * np.sqrt(0.3),
                     synth.gaussian((n,), (qmin,), (qmax,), (q0,), (p0,), (sigma,)) * np.sqrt(0.7)])
    pr = _problem_1d(V, psi0, n, qmin, qmax, m)
    assert O.kinetic_energy(pr, psi0) == pytest.approx((p0 ** 2 + 0.5 / sigma ** 2) / (2 * m), rel=1e-12)
    assert O.potential_energy(pr, psi0) == pytest.approx(0.5 * k * (q0 ** 2 + sigma ** 2 / 2) + 0.7 * 0.25,
                                                        rel=1e-12)
    pops = O.populations(pr, psi0)
    assert pops == pytest.approx([0.3, 0.7], abs=1e-14)
    assert O.norm(pr, psi0) ** 2 == pytest.approx(1.0, abs=1e-14)
