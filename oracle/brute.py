"""Exact propagation on tiny grids by dense diagonalisation (oracle).

Eq. (exact_evol_op): U(t) = exp(-i H t).  On the grid, H = I_S (x) K + V with
K = F^{-1} diag(T(p)) F the Fourier-grid kinetic matrix (the same on every
surface) and V block-diagonal in q with the S x S potential at every point.
H is Hermitian; U(t) = W exp(-i Lambda t) W^dagger from LAPACK's Hermitian
eigensolver (a library step).  Only for S * prod(n) of a few hundred.
"""
from __future__ import annotations

import numpy as np

from . import operators


def grid_hamiltonian(problem) -> np.ndarray:
    n = tuple(problem.n)
    P = int(np.prod(n))
    S = problem.S
    T = operators.kinetic_energy(n, problem.qmin, problem.qmax, problem.mass).reshape(-1)
    # D-dimensional DFT matrix as a Kronecker product of 1-D ones
    F = np.ones((1, 1), dtype=np.complex128)
    for d in range(len(n)):
        j = np.arange(n[d])
        Fd = np.exp(-2j * np.pi * np.outer(j, j) / n[d])
        F = np.kron(F, Fd)
    K = (np.conj(F.T) / P) @ (T[:, None] * F)
    Vf = operators.unpack_potential(np.asarray(problem.V, dtype=np.float64), S).reshape(S, S, P)
    H = np.zeros((S * P, S * P), dtype=np.complex128)
    for s in range(S):
        H[s * P:(s + 1) * P, s * P:(s + 1) * P] += K
    for r in range(S):
        for c in range(S):
            H[r * P + np.arange(P), c * P + np.arange(P)] += Vf[r, c]
    return H


def exact_propagate(problem, psi, t: float) -> np.ndarray:
    H = grid_hamiltonian(problem)
    H = 0.5 * (H + np.conj(H.T))
    lam, W = np.linalg.eigh(H)
    v = psi.reshape(-1)
    out = W @ (np.exp(-1j * lam * t) * (np.conj(W.T) @ v))
    return out.reshape(psi.shape)
