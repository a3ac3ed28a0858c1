"""Pins of the oracle's inner product and symplectic two-form (Sec. II A)
against closed forms.

The overlap of two complex Gaussians has a closed form from the Gaussian
integral  int exp(-A q^2 + B q + C) dq = sqrt(pi / A) exp(B^2 / (4A) + C)
(Re A > 0).  On a periodic grid that is wide and fine enough, the grid sum
sum_q f(q) dq of a smooth, decayed integrand equals the integral to round-off
(the error of the trapezoidal rule for such functions is exponentially small),
so the oracle's <psi|phi> must reproduce the closed form to ~1e-14.

The test cases are chosen so that each plausible slip fails one of them:
the complex conjugate on the wrong argument flips the sign of the imaginary
part (momenta differ, so Im <psi|phi> != 0); a missing cell volume dV is off
by the factor dV != 1; a dropped surface, a wrong surface amplitude or a
mis-summed axis changes the product/sum structure; omega = -2 Im<psi|phi>
fixes value, sign and the factor 2.
"""
import cmath
import math

import numpy as np
import pytest

import synth
from oracle import observables as O


def gauss_1d(q, q0, p0, sigma):
    """exp(-(q-q0)^2/(2 sigma^2) + i p0 (q-q0)), unnormalised."""
    return np.exp(-((q - q0) ** 2) / (2.0 * sigma ** 2) + 1j * p0 * (q - q0))


def overlap_1d(qa, pa, sa, qb, pb, sb):
    """int conj(g_a(q)) g_b(q) dq for the unnormalised Gaussians above,
    by the Gaussian integral (written out independently of the oracle)."""
    A = 1.0 / (2.0 * sa ** 2) + 1.0 / (2.0 * sb ** 2)
    B = qa / sa ** 2 + qb / sb ** 2 + 1j * (pb - pa)
    C = -qa ** 2 / (2.0 * sa ** 2) - qb ** 2 / (2.0 * sb ** 2) + 1j * pa * qa - 1j * pb * qb
    return cmath.sqrt(math.pi / A) * cmath.exp(B * B / (4.0 * A) + C)


def _problem(n, qmin, qmax, S):
    D = len(n)
    return synth.Problem(n=tuple(n), qmin=tuple(qmin), qmax=tuple(qmax), mass=tuple([1.0] * D), S=S,
                         V=np.zeros((S * (S + 1) // 2,) + tuple(n)),
                         psi0=np.zeros((S,) + tuple(n), complex))


def _state(pr, amps, params):
    """psi_s = amps[s] * prod_d g(q_d; params[s][d]) on the grid of pr."""
    Q = synth.mesh(pr.n, pr.qmin, pr.qmax)
    psi = np.zeros((pr.S,) + tuple(pr.n), complex)
    for s in range(pr.S):
        f = np.ones(Q[0].shape, complex)
        for d in range(pr.D):
            q0, p0, sig = params[s][d]
            f = f * gauss_1d(Q[d], q0, p0, sig)
        psi[s] = amps[s] * f
    return psi


def _closed(amps_a, pa, amps_b, pb):
    tot = 0.0 + 0.0j
    for s in range(len(amps_a)):
        prod = 1.0 + 0.0j
        for d in range(len(pa[s])):
            prod *= overlap_1d(*pa[s][d], *pb[s][d])
        tot += np.conj(amps_a[s]) * amps_b[s] * prod
    return complex(tot)


def test_inner_one_surface_1d_displaced_gaussians():
    pr = _problem((256,), (-12.0,), (12.0,), 1)
    ga = [[(0.4, 0.3, 0.9)]]
    gb = [[(-0.4, 1.5, 1.0)]]
    psi, phi = _state(pr, [1.0], ga), _state(pr, [1.0], gb)
    ref = _closed([1.0], ga, [1.0], gb)
    got = O.inner(pr, psi, phi)
    assert abs(ref.imag) > 0.1 and abs(ref.real) > 0.1  # both parts carry information
    assert abs(got - ref) <= 1e-13 * abs(ref)
    # conjugate symmetry and the two-form, value and sign
    assert abs(O.inner(pr, phi, psi) - np.conj(ref)) <= 1e-13 * abs(ref)
    assert O.symplectic_form(pr, psi, phi) == pytest.approx(-2.0 * ref.imag, rel=1e-13)
    assert O.symplectic_form(pr, phi, psi) == pytest.approx(2.0 * ref.imag, rel=1e-13)


def test_norm_and_populations_closed_form():
    # ||g||^2 = sqrt(pi) sigma per axis for the unnormalised Gaussian
    pr = _problem((64, 128), (-8.0, -9.0), (8.0, 9.0), 2)
    params = [[(0.3, 0.5, 0.9), (-0.2, 1.0, 1.2)], [(-1.0, -0.3, 0.7), (0.8, 0.2, 1.0)]]
    amps = [0.6 - 0.2j, 1.3j]
    psi = _state(pr, amps, params)
    pops = [abs(amps[s]) ** 2 * np.prod([math.sqrt(math.pi) * params[s][d][2] for d in range(2)])
            for s in range(2)]
    assert O.populations(pr, psi) == pytest.approx(pops, rel=1e-13)
    assert O.norm(pr, psi) == pytest.approx(math.sqrt(sum(pops)), rel=1e-13)


@pytest.mark.parametrize("n,extent", [((48, 64, 40), (9.0, 10.0, 8.0)), ((32, 32), (7.0, 7.5))])
def test_inner_multisurface_multid(n, extent):
    D = len(n)
    S = 3
    rng = np.random.default_rng(17 + D)
    pr = _problem(n, [-e for e in extent], list(extent), S)
    pa = [[(rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(0.7, 1.1)) for _ in range(D)] for _ in range(S)]
    pb = [[(rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(0.7, 1.1)) for _ in range(D)] for _ in range(S)]
    aa = [complex(rng.normal(), rng.normal()) for _ in range(S)]
    ab = [complex(rng.normal(), rng.normal()) for _ in range(S)]
    psi, phi = _state(pr, aa, pa), _state(pr, ab, pb)
    ref = _closed(aa, pa, ab, pb)
    got = O.inner(pr, psi, phi)
    assert abs(got - ref) <= 1e-13 * max(1.0, abs(ref))
    assert O.symplectic_form(pr, psi, phi) == pytest.approx(-2.0 * ref.imag, rel=1e-12, abs=1e-14)
    # the cell volume is part of the measure: it is far from 1 here
    dV = np.prod([2 * e / m for e, m in zip(extent, n)])
    assert abs(dV - 1.0) > 0.1


def test_inner_orthogonal_surfaces_vanish():
    # states on different surfaces are orthogonal, whatever their shapes
    pr = _problem((128,), (-10.0,), (10.0,), 2)
    psi = _state(pr, [1.0, 0.0], [[(0.0, 0.0, 1.0)], [(0.0, 0.0, 1.0)]])
    phi = _state(pr, [0.0, 1.0], [[(0.0, 0.0, 1.0)], [(0.0, 0.0, 1.0)]])
    assert O.inner(pr, psi, phi) == 0.0
    assert O.symplectic_form(pr, psi, phi) == 0.0


def test_phase_at_density_maximum_closed_forms():
    # a Gaussian of known global phase: the density peaks at its centre
    pr = _problem((256,), (-10.0,), (10.0,), 2)
    q = synth.axis_points(256, -10.0, 10.0)
    dq = 20.0 / 256
    q0 = q[137]  # centre on a grid point
    psi = np.zeros((2, 256), complex)
    psi[0] = np.exp(1j * 0.7) * gauss_1d(q, q0, 0.0, 0.9)
    psi[1] = np.exp(-1j * 2.9) * 0.3 * gauss_1d(q, q[40], 1.3, 0.5)  # momentum: phase 0 at the centre
    idx, ph = O.phase_at_density_maximum(pr, psi)
    assert list(idx) == [137, 40]
    assert ph[0] == pytest.approx(0.7, abs=1e-15)
    assert ph[1] == pytest.approx(-2.9, abs=1e-15)
    # a coherent state of a harmonic oscillator (m = 1, omega = 1, sigma = 1,
    # p0 = 0) after time t: psi = pi^-1/4 exp(-(q - q0 cos t)^2 / 2
    # - i (q q0 sin t - q0^2 sin 2t / 4) - i t / 2); at the density maximum
    # q = q0 cos t the phase is -(q0^2 sin 2t)/4 - t/2 (mod 2 pi)
    t, q0c = 0.8, 1.5
    qc = q0c * np.cos(t)
    kk = int(np.argmin(np.abs(q - qc)))
    qg = q - (q[kk] - qc)  # shift the grid so that qc is a grid point
    coh = np.pi ** -0.25 * np.exp(-(qg - qc) ** 2 / 2 - 1j * (qg * q0c * np.sin(t) - q0c ** 2 * np.sin(2 * t) / 4)
                                  - 1j * t / 2)
    psi2 = np.stack([coh, np.zeros_like(coh)])
    idx2, ph2 = O.phase_at_density_maximum(pr, psi2)
    want = np.angle(np.exp(1j * (-(q0c ** 2) * np.sin(2 * t) / 4 - t / 2)))
    assert idx2[0] == kk
    assert ph2[0] == pytest.approx(want, abs=1e-14)
    assert dq > 0
