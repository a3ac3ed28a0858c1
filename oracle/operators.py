"""Grids and the two elementary evolution operators (oracle).

* Kinetic: the Hamiltonian of Eq. (diab_mol_ham) has T(p) = p^T m^{-1} p / 2
  with a diagonal mass matrix, the same on every surface; U_T(t) =
  exp(-i t T(p)) is diagonal in the momentum representation (Sec. II G).
* Potential: V(q) is a real symmetric S x S matrix at each grid point;
  U_V(t) = exp(-i t V(q)) is an S x S unitary at each point (Sec. II H).
  For S = 2 one Jacobi rotation diagonalises V exactly, which gives the
  closed form used by ``expm_potential_2x2``; the general path diagonalises
  with LAPACK's symmetric eigensolver (a library step) and exponentiates the
  eigenvalues.

hbar = 1 throughout (atomic units).
"""
from __future__ import annotations

import numpy as np


def axis_positions(n: int, qmin: float, qmax: float) -> np.ndarray:
    """q_k = qmin + k dq, dq = (qmax - qmin)/n, k = 0..n-1 (periodic grid,
    right endpoint excluded; App. B)."""
    dq = (qmax - qmin) / n
    return qmin + dq * np.arange(n, dtype=np.float64)


def axis_momenta(n: int, qmin: float, qmax: float) -> np.ndarray:
    """Momenta conjugate to the FFT index: p_k = 2 pi k / (n dq) for k < n/2,
    2 pi (k - n)/(n dq) otherwise (the Nyquist index n/2 maps to -n/2)."""
    dq = (qmax - qmin) / n
    k = np.arange(n, dtype=np.float64)
    k = np.where(k < n // 2, k, k - n)
    return 2.0 * np.pi * k / (n * dq)


def kinetic_energy(n, qmin, qmax, mass) -> np.ndarray:
    """T(p) = sum_d p_d^2 / (2 m_d) on the momentum grid (Eq. diab_mol_ham)."""
    D = len(n)
    out = np.zeros(tuple(n), dtype=np.float64)
    for d in range(D):
        p = axis_momenta(n[d], qmin[d], qmax[d])
        shape = [1] * D
        shape[d] = n[d]
        out = out + (p * p / (2.0 * mass[d])).reshape(shape)
    return out


def kinetic_phase(T: np.ndarray, t: float) -> np.ndarray:
    """exp(-i t T(p)) (Sec. II G)."""
    return np.exp(-1j * t * T)


def unpack_potential(Vp: np.ndarray, S: int) -> np.ndarray:
    """Packed upper triangle [S(S+1)/2, *grid] -> full symmetric [S, S, *grid]."""
    full = np.empty((S, S) + Vp.shape[1:], dtype=np.float64)
    k = 0
    for r in range(S):
        for c in range(r, S):
            full[r, c] = Vp[k]
            full[c, r] = Vp[k]
            k += 1
    return full


def expm_potential(Vfull: np.ndarray, t: float) -> np.ndarray:
    """exp(-i t V(q)) for every grid point, any S, by eigendecomposition
    V = W diag(lam) W^T: U = W diag(exp(-i t lam)) W^T (Sec. II H)."""
    S = Vfull.shape[0]
    grid = Vfull.shape[2:]
    M = np.moveaxis(Vfull.reshape(S, S, -1), -1, 0)          # [P, S, S]
    lam, W = np.linalg.eigh(M)
    ph = np.exp(-1j * t * lam)                                  # [P, S]
    U = np.einsum("pik,pk,pjk->pij", W, ph, W)
    return np.moveaxis(U, 0, -1).reshape((S, S) + grid)


def expm_potential_2x2(Vfull: np.ndarray, t: float) -> np.ndarray:
    """Closed form for S = 2 (one Jacobi rotation is exact, Sec. II H).
    With V = v0 1 + vx sigma_x + vz sigma_z and r = sqrt(vx^2 + vz^2),
    exp(-i t V) = exp(-i t v0) [cos(r t) 1 - i sin(r t) (vx sigma_x + vz sigma_z)/r];
    at r = 0 the bracket is the identity."""
    v11, v12, v22 = Vfull[0, 0], Vfull[0, 1], Vfull[1, 1]
    v0 = 0.5 * (v11 + v22)
    vz = 0.5 * (v11 - v22)
    vx = v12
    r = np.sqrt(vx * vx + vz * vz)
    c = np.cos(r * t)
    # sin(r t)/r with the r -> 0 limit t
    with np.errstate(invalid="ignore", divide="ignore"):
        sr = np.where(r > 0, np.sin(r * t) / np.where(r > 0, r, 1.0), t)
    g = np.exp(-1j * t * v0)
    U = np.empty((2, 2) + v11.shape, dtype=np.complex128)
    U[0, 0] = g * (c - 1j * sr * vz)
    U[1, 1] = g * (c + 1j * sr * vz)
    U[0, 1] = g * (-1j * sr * vx)
    U[1, 0] = U[0, 1]
    return U


def apply_potential(U: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """psi_r(q) <- sum_c U_rc(q) psi_c(q) at every grid point."""
    return np.einsum("rc...,c...->r...", U, psi)
