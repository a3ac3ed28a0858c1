"""Split-operator propagation (oracle).

A general split-operator step (Sec. II E) is
U(dt) = U_B(b_N dt) U_A(a_N dt) ... U_B(b_1 dt) U_A(a_1 dt),
so U_A(a_1 dt) acts first.  The VTV algorithm, Eq. (so_VTV), is the
second-order case with A = V, B = T and a = (1/2, 1/2), b = (1, 0); TVT,
Eq. (so_TVT), swaps the roles (A = T, B = V).  The first-order VT algorithm,
Eq. (so_VT), applies T first (A = T, B = V, a = b = 1); TV, Eq. (so_TV),
applies V first.  Compositions (Sec. II D) and pruning (Sec. II F) only change
the coefficient lists.  The kinetic action is taken in the momentum
representation reached by an FFT of every surface over all grid axes, the
potential action in the position representation (Sec. II G).
"""
from __future__ import annotations

import numpy as np

from . import coefficients as C
from . import fourier, operators

VTV, TVT, VT, TV = "VTV", "TVT", "VT", "TV"


def action_sequence(elementary: str = VTV, order: int = 2, scheme: str = C.TRIPLE_JUMP,
                    pruned: bool = True, gammas=None):
    """Ordered list of (operator, coefficient) for one time step; the first
    entry acts first."""
    if elementary in (VT, TV):
        A, B = ("T", "V") if elementary == VT else ("V", "T")
        return [(A, 1.0), (B, 1.0)]
    sp = C.Splitting(order, scheme, pruned, gammas=gammas)
    A, B = ("V", "T") if elementary == VTV else ("T", "V")
    seq = []
    for j in range(len(sp.b)):
        seq.append((A, sp.a[j]))
        seq.append((B, sp.b[j]))
    if len(sp.a) > len(sp.b):
        seq.append((A, sp.a[-1]))
    return seq


class Propagator:
    """Applies an action sequence to psi[s, *grid] on one problem."""

    def __init__(self, problem, dft: bool = False, closed_form_2x2: bool = True):
        self.p = problem
        self.S = problem.S
        self.T = operators.kinetic_energy(problem.n, problem.qmin, problem.qmax, problem.mass)
        self.Vfull = operators.unpack_potential(np.asarray(problem.V, dtype=np.float64), self.S)
        self.dft = dft
        self.closed_form_2x2 = closed_form_2x2
        self._uv = {}
        self._ut = {}

    def potential_unitary(self, tau: float):
        if tau not in self._uv:
            if self.S == 2 and self.closed_form_2x2:
                self._uv[tau] = operators.expm_potential_2x2(self.Vfull, tau)
            else:
                self._uv[tau] = operators.expm_potential(self.Vfull, tau)
        return self._uv[tau]

    def kinetic_unitary(self, tau: float):
        if tau not in self._ut:
            self._ut[tau] = operators.kinetic_phase(self.T, tau)
        return self._ut[tau]

    def apply_V(self, psi, tau):
        return operators.apply_potential(self.potential_unitary(tau), psi)

    def apply_T(self, psi, tau):
        f = fourier.fftn_grid(psi, inverse=False, dft=self.dft)
        f = f * self.kinetic_unitary(tau)[None]
        return fourier.fftn_grid(f, inverse=True, dft=self.dft)

    def step(self, psi, seq, dt):
        for op, c in seq:
            psi = self.apply_V(psi, c * dt) if op == "V" else self.apply_T(psi, c * dt)
        return psi

    def run(self, psi, seq, dt, nsteps):
        psi = np.array(psi, dtype=np.complex128, copy=True)
        for _ in range(nsteps):
            psi = self.step(psi, seq, dt)
        return psi


def propagate(problem, t: float, dt: float, order: int = 2, scheme: str = C.TRIPLE_JUMP,
              elementary: str = VTV, pruned: bool = True, psi=None, gammas=None):
    """Propagate ``problem.psi0`` (or ``psi``) to time t with step dt;
    t/dt must be an integer.  ``gammas``: explicit composition coefficients
    in place of the recursive scheme."""
    nsteps = int(round(t / dt))
    if abs(nsteps * dt - t) > 1e-9 * max(1.0, abs(t)):
        raise ValueError("t must be an integer multiple of dt")
    prop = Propagator(problem)
    seq = action_sequence(elementary, order, scheme, pruned, gammas)
    return prop.run(problem.psi0 if psi is None else psi, seq, dt, nsteps)
