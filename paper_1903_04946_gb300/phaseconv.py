"""Convergence of the wavepacket phase (the phase study of Sec. III A).

Beside the wavefunction error, the paper follows how the phase of the
wavepacket converges with the time step.  Its definition is deferred to the
companion paper; this module reads it as the phase of each surface's
wavefunction at that surface's density maximum, arg psi_s(q*) with q* the grid
point of largest |psi_s|^2 (dso_phase_at_density_maximum).  For one model,
composition scheme and order, the propagation to t_f is repeated with
dt = t_f / 2^k, and the phase error at dt is |wrap(phase_dt - phase_ref)| with
the reference at the smallest step; a method of order n gives errors falling
as dt^n until round-off.

    python -m paper_1903_04946_gb300.phaseconv [--tf 2000] [--order 4] [--scheme triple_jump]

Prints one JSON document.
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import SCHEME_CODES, Context


def wrap(x):
    """Angle difference folded to (-pi, pi]."""
    return float(np.angle(np.exp(1j * x)))


def phases(problem, order, scheme, tf, k, device=0):
    """(indices, phases) per surface after propagating to tf with dt = tf / 2^k."""
    ctx = Context(problem, device=device, order=order,
                  scheme=SCHEME_CODES[scheme])
    try:
        ctx.propagate(tf, tf / 2 ** k)
        return ctx.phase_at_density_maximum()
    finally:
        ctx.close()


def study(problem=None, order=4, scheme="triple_jump", tf=2000.0, ks=(7, 8, 9, 10, 11), ref_k=14,
          surface=None, device=0):
    """Phase errors of one method at dt = tf / 2^k, k in ks, against the
    same method at tf / 2^ref_k, and the fitted convergence order."""
    import synth
    if problem is None:
        problem = synth.nai_like()
    ref_idx, ref_ph = phases(problem, order, scheme, tf, ref_k, device)
    s = 0 if surface is None else surface  # the surface the packet starts on by default
    rows = []
    for k in ks:
        idx, ph = phases(problem, order, scheme, tf, k, device)
        rows.append({"k": k, "dt": tf / 2 ** k, "index": int(idx[s]), "ref_index": int(ref_idx[s]),
                     "phase": float(ph[s]), "error": abs(wrap(ph[s] - ref_ph[s]))})
    ok = [r for r in rows if r["index"] == r["ref_index"] and r["error"] > 1e-12]
    slope = None
    if len(ok) >= 2:
        x = np.log([r["dt"] for r in ok])
        y = np.log([r["error"] for r in ok])
        slope = float(np.polyfit(x, y, 1)[0])
    return {"model": problem.name, "scheme": scheme, "order": order, "t_final": tf, "surface": s,
            "reference_k": ref_k, "rows": rows, "fitted_order": slope}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--tf", type=float, default=2000.0)
    ap.add_argument("--order", type=int, default=4)
    ap.add_argument("--scheme", default="triple_jump", choices=["triple_jump", "suzuki"])
    args = ap.parse_args()
    print(json.dumps(study(order=args.order, scheme=args.scheme, tf=args.tf)))


if __name__ == "__main__":
    main()
