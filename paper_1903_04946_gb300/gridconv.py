"""Exponential convergence with the grid density (the study of App. B).

A 1-D two-surface NaI-like model is propagated on grids of N = 2^8 .. 2^12
points.  Each doubling of N widens the range and refines the spacing by the
same factor sqrt(2): the grid starts at q = 3 bohr (the inner wall) and ends
at 3 + 27 sqrt(N / 1024), so N = 1024 is the standard [3, 30) grid.  Every
grid gets the same seeded model evaluated at its own points and the same
Gaussian packet.  Results on different grids are compared on the finest grid
by trigonometric interpolation of the coarser wavefunction: the Fourier
series that the coarse samples define (periodic over the coarse range) is
evaluated at the fine points inside the coarse range, and taken as zero
outside it.  Reported per N, at t = 0 and at t_f:

* the total error ||I_N psi_N - psi_ref|| (grid L2 norm on the finest grid,
  summed over surfaces);
* the representation ("integration") error ||I_N R_N psi_ref - psi_ref||,
  where R_N samples the finest result at the N-grid points, so the grid acts
  only after the propagation;
* their ratio.

Propagation runs in the library (VTV, Suzuki order 6, dt = t_f / 2^7); the
interpolation is plain numpy on the host.

    python -m paper_1903_04946_gb300.gridconv [--tf 2000] [--nmax 4096]

prints one JSON document.
"""
from __future__ import annotations

import argparse
import json

import numpy as np

Q0, R1024 = 3.0, 27.0


def grid_range(N: int):
    return Q0, Q0 + R1024 * np.sqrt(N / 1024.0)


def trig_interpolate(f, a, b, x, chunk=1024):
    """Evaluate at the points x the trigonometric interpolant of samples f
    (last axis) taken at a + j (b - a) / N, j = 0..N-1, periodic over
    [a, b).  Frequencies -N/2 .. N/2-1; points outside [a, b) give zero."""
    f = np.asarray(f, dtype=np.complex128)
    N = f.shape[-1]
    c = np.fft.fft(f, axis=-1) / N
    k = np.fft.fftfreq(N, d=1.0 / N)              # integer frequencies, -N/2 .. N/2-1
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros(f.shape[:-1] + x.shape, dtype=np.complex128)
    inside = (x >= a) & (x < b)
    xi = x[inside]
    vals = np.empty(f.shape[:-1] + xi.shape, dtype=np.complex128)
    for s in range(0, xi.size, chunk):
        ph = np.exp(2j * np.pi * np.outer(xi[s:s + chunk] - a, k) / (b - a))   # [m, N]
        vals[..., s:s + chunk] = c @ ph.T
    out[..., inside] = vals
    return out


def l2(f, dq):
    return float(np.sqrt(np.sum(np.abs(f) ** 2) * dq))


def study(tf=2000.0, nmax=4096, nmin=256, k=7, seed=1903, order=6):
    import synth
    from . import DSO_SUZUKI, Context, dso_set_scheme
    Ns = [n for n in (256, 512, 1024, 2048, 4096, 8192) if nmin <= n <= nmax]
    dt = tf / 2 ** k
    res = {}
    for N in Ns:
        a, b = grid_range(N)
        pr = synth.nai_like(seed=seed, N=N, qmin=a, qmax=b)
        ctx = Context(pr, order=order, scheme=DSO_SUZUKI)
        ctx.propagate(tf, dt)
        res[N] = (a, b, pr.psi0, ctx.psi())
        ctx.close()
    a_r, b_r, psi0_r, psit_r = res[Ns[-1]]
    Nr = Ns[-1]
    dq = (b_r - a_r) / Nr
    xr = a_r + dq * np.arange(Nr)
    rows = []
    for N in Ns[:-1]:
        a, b, psi0, psit = res[N]
        xs = a + (b - a) / N * np.arange(N)
        row = {"N": N, "range": [a, b]}
        for label, coarse, ref in (("initial", psi0, psi0_r), ("final", psit, psit_r)):
            total = l2(trig_interpolate(coarse, a, b, xr) - ref, dq)
            rep = trig_interpolate(trig_interpolate(ref, a_r, b_r, xs), a, b, xr)
            integ = l2(rep - ref, dq)
            row[label] = {"total_error": total, "representation_error": integ,
                          "ratio": integ / total if total > 0 else None}
        rows.append(row)
    return {"model": f"NaI-like 1-D two-surface, seed {seed}; range [3, 3 + 27 sqrt(N/1024)) bohr",
            "method": f"VTV Suzuki order {order}, dt = t_f/2^{k}", "t_final": tf, "reference_N": Nr,
            "grids": rows}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--tf", type=float, default=2000.0)
    ap.add_argument("--nmax", type=int, default=4096)
    args = ap.parse_args()
    print(json.dumps(study(args.tf, args.nmax)))


if __name__ == "__main__":
    main()
