"""Observables of a multi-surface wavepacket (oracle).

Sec. II A defines the norm, the inner product, the symplectic two-form
omega(psi, phi) = -2 hbar Im<psi|phi> and the energy <psi|H|psi>; Sec. III A
also follows the phase of the wavepacket at its density maximum.  On the grid
the inner product is <psi|phi> = sum_s sum_q conj(psi_s(q)) phi_s(q) dV with
dV the product of the grid spacings.  <T> is evaluated in the momentum
representation: with the unnormalised forward FFT, sum_q |psi|^2 =
(1/P) sum_k |psi~_k|^2 (Parseval), so <T> = dV/P sum_k T(p_k) |psi~_k|^2.
"""
from __future__ import annotations

import numpy as np

from . import fourier, operators


def cell_volume(problem) -> float:
    return float(np.prod([(problem.qmax[d] - problem.qmin[d]) / problem.n[d]
                          for d in range(len(problem.n))]))


def inner(problem, psi, phi) -> complex:
    return complex(np.sum(np.conj(psi) * phi) * cell_volume(problem))


def norm(problem, psi) -> float:
    return float(np.sqrt(np.sum(np.abs(psi) ** 2) * cell_volume(problem)))


def populations(problem, psi) -> np.ndarray:
    axes = tuple(range(1, psi.ndim))
    return np.sum(np.abs(psi) ** 2, axis=axes) * cell_volume(problem)


def symplectic_form(problem, psi, phi) -> float:
    return -2.0 * inner(problem, psi, phi).imag


def potential_energy(problem, psi) -> float:
    Vf = operators.unpack_potential(np.asarray(problem.V, dtype=np.float64), problem.S)
    Vpsi = np.einsum("rc...,c...->r...", Vf, psi)
    return float(np.real(np.sum(np.conj(psi) * Vpsi)) * cell_volume(problem))


def kinetic_energy(problem, psi) -> float:
    T = operators.kinetic_energy(problem.n, problem.qmin, problem.qmax, problem.mass)
    f = fourier.fftn_grid(psi)
    P = int(np.prod(problem.n))
    return float(np.sum(T[None] * np.abs(f) ** 2) * cell_volume(problem) / P)


def energy(problem, psi) -> float:
    return kinetic_energy(problem, psi) + potential_energy(problem, psi)


def phase_at_density_maximum(problem, psi):
    """Phase of each surface's wavefunction where its density is largest
    (the wavepacket-phase observable of the phase-convergence study, Sec.
    III A; read as arg psi_s(q*) with q* the grid point of largest
    |psi_s(q)|^2, the first such point in storage order on a tie).  Returns
    (flat indices q*, phases in (-pi, pi]) per surface."""
    S = psi.shape[0]
    flat = psi.reshape(S, -1)
    idx = np.argmax(np.abs(flat) ** 2, axis=1)
    vals = flat[np.arange(S), idx]
    return idx, np.angle(vals)


def l2_error(problem, psi, ref) -> float:
    """||psi - ref|| with the grid measure, summed over surfaces."""
    return float(np.sqrt(np.sum(np.abs(psi - ref) ** 2) * cell_volume(problem)))


def rel_l2(psi, ref) -> float:
    """Relative L2 difference ||psi - ref|| / ||ref|| (measure cancels)."""
    return float(np.sqrt(np.sum(np.abs(psi - ref) ** 2) / np.sum(np.abs(ref) ** 2)))
