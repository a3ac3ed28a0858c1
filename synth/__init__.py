"""Seeded synthetic inputs for diabatic wavepacket propagation.

This module is the one place that both the CUDA library's tests/benchmark and
the CPU oracle draw their inputs from.  It only *generates* inputs -- grids,
diabatic potential matrices sampled on the grid, masses and initial
wavepackets -- and holds none of the propagation arithmetic (no splitting
coefficients, no Fourier transforms, no matrix exponentials).

The models follow the shapes of the paper's two numerical examples (Sec. III):
a one-dimensional two-surface "NaI-like" model (Sec. III A) and a
three-dimensional three-surface vibronic-coupling "pyrazine-like" model
(Sec. III B).  The literature parameters of both models are not available, so
every parameter is drawn from a seeded range; the recipes are stated in each
generator's docstring.

Conventions shared by both sides:

* grid axis d has ``n[d]`` points ``q_k = qmin[d] + k * (qmax[d]-qmin[d])/n[d]``,
  ``k = 0..n[d]-1`` (periodic, right endpoint excluded);
* the wavefunction is ``psi[s, i0, ..., i_{D-1}]``, complex128, surface-major,
  last axis contiguous;
* the potential is passed packed: ``V[k, i0, ...]`` for the upper-triangle
  pairs ``(r, c), r <= c`` in row-major order, e.g. ``(0,0), (0,1), (1,1)``
  for S = 2 and ``(0,0), (0,1), (0,2), (1,1), (1,2), (2,2)`` for S = 3;
* atomic units, hbar = 1.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Problem:
    """One propagation input: grid, masses, packed potential and psi0."""

    n: tuple                      # points per axis
    qmin: tuple                   # left grid edge per axis
    qmax: tuple                   # right grid edge per axis (excluded)
    mass: tuple                   # diagonal mass matrix, one entry per axis
    S: int                        # number of electronic surfaces
    V: np.ndarray                 # [S(S+1)/2, *n] float64, packed upper triangle
    psi0: np.ndarray              # [S, *n] complex128
    name: str = ""
    params: dict = field(default_factory=dict)

    @property
    def D(self) -> int:
        return len(self.n)

    @property
    def points(self) -> int:
        return int(np.prod(self.n))


def packed_index(r: int, c: int, S: int) -> int:
    """Position of the pair (r, c) in the packed upper-triangle layout."""
    if r > c:
        r, c = c, r
    return r * S - r * (r - 1) // 2 + (c - r)


def axis_points(n: int, qmin: float, qmax: float) -> np.ndarray:
    """Grid positions of one periodic axis (right endpoint excluded)."""
    return qmin + np.arange(n, dtype=np.float64) * ((qmax - qmin) / n)


def mesh(n, qmin, qmax):
    """Position arrays of a D-dimensional grid, ``indexing='ij'``."""
    axes = [axis_points(n[d], qmin[d], qmax[d]) for d in range(len(n))]
    return np.meshgrid(*axes, indexing="ij")


def gaussian(n, qmin, qmax, q0, p0, sigma):
    """Product Gaussian exp(-(q-q0)^2/(2 sigma^2) + i p0 (q-q0)), normalised
    numerically on the grid (sum |psi|^2 * dV = 1)."""
    Q = mesh(n, qmin, qmax)
    arg = np.zeros(Q[0].shape, dtype=np.complex128)
    for d in range(len(n)):
        arg += -((Q[d] - q0[d]) ** 2) / (2.0 * sigma[d] ** 2) + 1j * p0[d] * (Q[d] - q0[d])
    g = np.exp(arg)
    dV = float(np.prod([(qmax[d] - qmin[d]) / n[d] for d in range(len(n))]))
    return g / np.sqrt(np.sum(np.abs(g) ** 2) * dV)


# ---------------------------------------------------------------------------
# 1-D two-surface NaI-like model (shape of Sec. III A)
# ---------------------------------------------------------------------------

def nai_like(seed: int = 1903, N: int = 1024, qmin: float = 3.0, qmax: float = 30.0,
             mass: float = 1.5e4) -> Problem:
    """Seeded one-dimensional two-surface diabatic model.

    Surface 1 (index 0) is an ionic curve ``Delta + A exp(-q/rho) - 1/q``;
    surface 2 (index 1) a Morse covalent curve ``De (1 - exp(-beta (q-qe)))^2``;
    the coupling is a Gaussian ``c exp(-(q-qx)^2 / (2 w^2))`` centred on the
    crossing point qx.  Draws (uniform): De in [0.015, 0.03], beta in [0.5, 0.7],
    qe in [4.5, 5.5], rho in [0.6, 0.9], ionic minimum qm in [4.5, 6]
    (A = rho exp(qm/rho)/qm^2 puts the minimum there), crossing qx in [7, 9]
    (Delta chosen so the two curves meet at qx), c in [1e-3, 3e-3] Ha,
    w in [0.5, 1.5].  The initial Gaussian (p0 = 0, width sigma in
    [0.1, 0.25]) sits on surface 1 at the inner wall point q0 < qm where
    V11(q0) = V11(qx) + delta, delta in [0.002, 0.01], so that it swings
    through the crossing region.
    """
    rng = np.random.default_rng(seed)
    De = rng.uniform(0.015, 0.03)
    beta = rng.uniform(0.5, 0.7)
    qe = rng.uniform(4.5, 5.5)
    rho = rng.uniform(0.6, 0.9)
    qm = rng.uniform(4.5, 6.0)
    qx = rng.uniform(7.0, 9.0)
    c = rng.uniform(1e-3, 3e-3)
    w = rng.uniform(0.5, 1.5)
    sigma = rng.uniform(0.1, 0.25)
    delta = rng.uniform(0.002, 0.01)
    A = rho * np.exp(qm / rho) / qm ** 2

    def morse(q):
        return De * (1.0 - np.exp(-beta * (q - qe))) ** 2

    Delta = morse(qx) - A * np.exp(-qx / rho) + 1.0 / qx

    def ionic(q):
        return Delta + A * np.exp(-q / rho) - 1.0 / q

    # inner wall point with V11(q0) = V11(qx) + delta, by bisection on (qmin, qm)
    target = ionic(qx) + delta
    lo, hi = qmin, qm
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if ionic(mid) > target:
            lo = mid
        else:
            hi = mid
    q0 = 0.5 * (lo + hi)

    q = axis_points(N, qmin, qmax)
    V = np.empty((3, N), dtype=np.float64)
    V[0] = ionic(q)
    V[1] = c * np.exp(-((q - qx) ** 2) / (2.0 * w ** 2))
    V[2] = morse(q)
    psi0 = np.zeros((2, N), dtype=np.complex128)
    psi0[0] = gaussian((N,), (qmin,), (qmax,), (q0,), (0.0,), (sigma,))
    return Problem(n=(N,), qmin=(qmin,), qmax=(qmax,), mass=(mass,), S=2, V=V,
                   psi0=psi0, name=f"nai_like_N{N}",
                   params=dict(seed=seed, De=De, beta=beta, qe=qe, rho=rho, qm=qm,
                               qx=qx, c=c, w=w, sigma=sigma, q0=q0, A=A, Delta=Delta))


# ---------------------------------------------------------------------------
# 3-D three-surface pyrazine-like vibronic-coupling model (shape of Sec. III B)
# ---------------------------------------------------------------------------

def pyrazine_like(seed: int = 1904, n=(64, 64, 64), S: int = 3, q_extent: float = 7.0,
                  start_surface: int = 1, omega=None) -> Problem:
    """Seeded linear-plus-quadratic vibronic-coupling model in dimensionless
    normal coordinates.

    Mode frequencies omega_i ~ U[0.005, 0.02]; mass m_i = 1/omega_i so that the
    kinetic energy is sum_i omega_i p_i^2 / 2 and the reference potential
    sum_i omega_i q_i^2 / 2 (on every surface).  Surface 1 (index 0) is
    uncoupled.  Surfaces s >= 2 get vertical energies E_s (E_2 in
    [0.12, 0.15], each next one 0.02-0.04 higher), linear shifts
    kappa_i^(s) ~ U[-0.01, 0.01], diagonal quadratic terms
    gamma_i^(s) ~ U[-0.002, 0.002], and neighbouring excited surfaces are
    coupled by lambda q_c with lambda ~ U[0.005, 0.01] and q_c the last mode.
    The grid is [-q_extent, q_extent) on every axis.  psi0 is the ground
    vibrational state (sigma = 1, q0 = p0 = 0) placed on ``start_surface``.
    ``omega`` fixes the frequencies (and so the masses) instead of drawing
    them; the other draws are unchanged.
    """
    rng = np.random.default_rng(seed)
    D = len(n)
    drawn = rng.uniform(0.005, 0.02, size=D)
    omega = drawn if omega is None else np.asarray(omega, dtype=np.float64)
    E = np.zeros(S)
    if S > 1:
        E[1] = rng.uniform(0.12, 0.15)
        for s in range(2, S):
            E[s] = E[s - 1] + rng.uniform(0.02, 0.04)
    kappa = rng.uniform(-0.01, 0.01, size=(S, D))
    kappa[0] = 0.0
    gam = rng.uniform(-0.002, 0.002, size=(S, D))
    gam[0] = 0.0
    lam = rng.uniform(0.005, 0.01, size=max(S - 2, 0))
    qmin = tuple([-q_extent] * D)
    qmax = tuple([q_extent] * D)
    Q = mesh(n, qmin, qmax)
    V0 = np.zeros(Q[0].shape)
    for i in range(D):
        V0 += 0.5 * omega[i] * Q[i] ** 2
    V = np.zeros((S * (S + 1) // 2,) + tuple(n))
    for s in range(S):
        diag = V0 + E[s]
        for i in range(D):
            diag = diag + kappa[s, i] * Q[i] + gam[s, i] * Q[i] ** 2
        V[packed_index(s, s, S)] = diag
    for s in range(1, S - 1):
        V[packed_index(s, s + 1, S)] = lam[s - 1] * Q[D - 1]
    psi0 = np.zeros((S,) + tuple(n), dtype=np.complex128)
    psi0[start_surface] = gaussian(n, qmin, qmax, [0.0] * D, [0.0] * D, [1.0] * D)
    return Problem(n=tuple(n), qmin=qmin, qmax=qmax, mass=tuple(1.0 / omega), S=S, V=V,
                   psi0=psi0, name="pyrazine_like_" + "x".join(map(str, n)),
                   params=dict(seed=seed, omega=omega, E=E, kappa=kappa, gamma=gam, lam=lam))


# ---------------------------------------------------------------------------
# Generic seeded models for tests (any D, S)
# ---------------------------------------------------------------------------

def random_coupled(seed: int, n, S: int, extent: float = 6.0, mass=None,
                   coupling: float = 0.02) -> Problem:
    """A smooth random coupled model of any dimension: harmonic diagonals with
    seeded shifts and offsets, and seeded linear-plus-Gaussian couplings
    between every pair of surfaces.  psi0 is a seeded complex Gaussian spread
    over all surfaces."""
    rng = np.random.default_rng(seed)
    D = len(n)
    qmin = tuple([-extent] * D)
    qmax = tuple([extent] * D)
    if mass is None:
        mass = tuple(rng.uniform(0.5, 2.0, size=D))
    Q = mesh(n, qmin, qmax)
    V = np.zeros((S * (S + 1) // 2,) + tuple(n))
    for r in range(S):
        for c in range(r, S):
            k = packed_index(r, c, S)
            if r == c:
                v = rng.uniform(-0.2, 0.2) * np.ones(Q[0].shape)
                for d in range(D):
                    v = v + 0.5 * rng.uniform(0.3, 1.0) * (Q[d] - rng.uniform(-1, 1)) ** 2
            else:
                v = coupling * rng.uniform(0.5, 1.0) * np.ones(Q[0].shape)
                for d in range(D):
                    v = v * np.exp(-((Q[d] - rng.uniform(-1, 1)) ** 2) / 4.0)
                    v = v + coupling * rng.uniform(-0.5, 0.5) * Q[d]
            V[k] = v
    psi0 = np.zeros((S,) + tuple(n), dtype=np.complex128)
    for s in range(S):
        amp = rng.uniform(0.2, 1.0) * np.exp(1j * rng.uniform(0, 2 * np.pi))
        psi0[s] = amp * gaussian(n, qmin, qmax, rng.uniform(-1.5, 1.5, size=D),
                                 rng.uniform(-1.0, 1.0, size=D), rng.uniform(0.7, 1.2, size=D))
    dV = float(np.prod([(qmax[d] - qmin[d]) / n[d] for d in range(D)]))
    psi0 /= np.sqrt(np.sum(np.abs(psi0) ** 2) * dV)
    return Problem(n=tuple(n), qmin=qmin, qmax=qmax, mass=tuple(mass), S=S, V=V, psi0=psi0,
                   name=f"random_coupled_{'x'.join(map(str, n))}_S{S}", params=dict(seed=seed))


def random_state(seed: int, like: Problem) -> np.ndarray:
    """A second seeded normalised state on the grid of ``like`` (for inner
    products)."""
    rng = np.random.default_rng(seed)
    D = like.D
    psi = np.zeros((like.S,) + tuple(like.n), dtype=np.complex128)
    for s in range(like.S):
        psi[s] = rng.uniform(0.2, 1.0) * gaussian(
            like.n, like.qmin, like.qmax,
            [like.qmin[d] + (like.qmax[d] - like.qmin[d]) * rng.uniform(0.35, 0.65) for d in range(D)],
            rng.uniform(-0.5, 0.5, size=D),
            [(like.qmax[d] - like.qmin[d]) * rng.uniform(0.03, 0.06) for d in range(D)])
    dV = float(np.prod([(like.qmax[d] - like.qmin[d]) / like.n[d] for d in range(D)]))
    return psi / np.sqrt(np.sum(np.abs(psi) ** 2) * dV)


# ---------------------------------------------------------------------------
# Mixed job stream for a serving loop (shape of the serving configuration)
# ---------------------------------------------------------------------------

SERVING_DT = {2: 2.0, 4: 10.0, 6: 20.0, 8: 40.0}


def serving_job(seed: int, max_points: int = 1 << 21, min_points: int = 1 << 8):
    """One seeded propagation request of the serving workload: D in {1, 2, 3},
    a power-of-two grid of min_points..max_points points per surface, S in
    {2, 3, 4} surfaces with harmonic diagonals in dimensionless normal
    coordinates (omega ~ U[0.005, 0.02], m = 1/omega) plus seeded linear
    couplings, a displaced Gaussian on surface 1, order in {2, 4, 6, 8}
    (triple jump), t ~ U[500, 5000] rounded to a multiple of the order's dt
    (SERVING_DT).  The grid's log2 size is drawn uniformly and its bits are
    spread at random over the D axes, each axis keeping at least 8 points
    (a D-dimensional grid therefore has at least 2^(3D) points).  Nothing is
    redrawn to fit an implementation: any axis length up to the full size
    can come out.  Returns (problem, order, t, dt)."""
    rng = np.random.default_rng(seed)
    D = int(rng.integers(1, 4))
    S = int(rng.integers(2, 5))
    lo = max(int(np.log2(min_points)), 3 * D)
    logp = int(rng.integers(lo, max(lo, int(np.log2(max_points))) + 1))
    parts = [3] * D
    for _ in range(logp - 3 * D):
        parts[int(rng.integers(0, D))] += 1
    n = tuple(2 ** p for p in parts)
    omega = rng.uniform(0.005, 0.02, size=D)
    extent = 7.0
    qmin, qmax = tuple([-extent] * D), tuple([extent] * D)
    Q = mesh(n, qmin, qmax)
    V = np.zeros((S * (S + 1) // 2,) + n)
    for r in range(S):
        for c in range(r, S):
            k = packed_index(r, c, S)
            if r == c:
                v = rng.uniform(0.0, 0.05) * np.ones(Q[0].shape) * r
                for d in range(D):
                    v = v + 0.5 * omega[d] * Q[d] ** 2 + rng.uniform(-0.01, 0.01) * Q[d]
            else:
                v = rng.uniform(0.002, 0.01) * Q[int(rng.integers(0, D))]
            V[k] = v
    psi0 = np.zeros((S,) + n, dtype=np.complex128)
    psi0[0] = gaussian(n, qmin, qmax, rng.uniform(-1.0, 1.0, size=D), [0.0] * D, [1.0] * D)
    order = int(rng.choice([2, 4, 6, 8]))
    dt = SERVING_DT[order]
    t = dt * max(1, int(round(rng.uniform(500.0, 5000.0) / dt)))
    pr = Problem(n=n, qmin=qmin, qmax=qmax, mass=tuple(1.0 / omega), S=S, V=V, psi0=psi0,
                 name=f"serving_{seed}", params=dict(seed=seed, omega=omega))
    return pr, order, t, dt


# ---------------------------------------------------------------------------
# Mixed batch: many 1-D two-surface packets on uneven grids plus 3-D
# three-surface instances on mixed 32/64 axes
# ---------------------------------------------------------------------------

BATCH_N_1D = (512, 1024, 2048, 4096, 8192)


def batch_jobs(seed: int = 1905, n_1d: int = 512, n_3d: int = 32):
    """Seeded mixed batch.  ``n_1d`` NaI-like packets with their own
    potentials and initial states, N cycling through 512..8192 on the common
    [3, 30) bohr range (mass 1.5e4); ``n_3d`` pyrazine-like instances whose
    axes are each 32 or 64 points (the 8 shapes in turn), with seeded
    couplings, vertical energies and shifts.  Instances of one shape share
    their mode frequencies (drawn once per shape), hence their masses, so
    that each shape advances as one batch.  Returns (jobs_1d, jobs_3d)."""
    jobs_1d = [nai_like(seed=seed * 1000 + i, N=BATCH_N_1D[i % len(BATCH_N_1D)]) for i in range(n_1d)]
    shapes = [(a, b, c) for a in (32, 64) for b in (32, 64) for c in (32, 64)]
    rng = np.random.default_rng(seed)
    omegas = {sh: rng.uniform(0.005, 0.02, size=3) for sh in shapes}
    jobs_3d = []
    for i in range(n_3d):
        sh = shapes[i % len(shapes)]
        jobs_3d.append(pyrazine_like(seed=seed * 1000 + 500 + i, n=sh, omega=omegas[sh]))
    return jobs_1d, jobs_3d


def group_batch(jobs):
    """Group jobs that can share one batched context (same grid, masses and
    surface count), keeping their order; returns a list of lists of indices."""
    groups = {}
    for i, pr in enumerate(jobs):
        key = (tuple(pr.n), tuple(pr.qmin), tuple(pr.qmax), tuple(np.round(pr.mass, 12)), pr.S)
        groups.setdefault(key, []).append(i)
    return list(groups.values())
