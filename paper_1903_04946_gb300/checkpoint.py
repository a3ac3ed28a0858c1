"""Checkpoint and resume of a propagation.

A checkpoint is the wavefunction (all jobs of a batch) with the number of
steps done, the step dt, and a digest of the composition it was made with:
the pruned coefficients a~, b~, their index arrays and the elementary
method.  Resuming checks the digest, so a run cannot continue with another
scheme by mistake, and loads psi into a context built for the same problem.

By default the uninterrupted run applies the last a~ action of a step and
the first of the next as one action with coefficient a~_last + a~_0
(dso_set_boundary_merge), where a run split at that boundary applies the two
in turn, so the results agree to round-off (tested to 1e-13).  With the
unmerged boundary (dso_set_boundary_merge(ctx, 0)) and the VTV method
resuming is exact: the split run applies the same operations in the same
order as the uninterrupted one, the last potential action of the first part
and then the first of the second; the tests check that the two results are
bitwise equal.  With TVT the uninterrupted run applies the two kinetic
actions of a step boundary between one forward and one inverse FFT, the
split run returns to position space in between, so the results agree to
round-off.

    ck = checkpoint.capture(ctx, order, scheme, elementary, steps_done, dt)
    checkpoint.save("run.npz", ck)
    ...
    ck = checkpoint.load("run.npz")
    checkpoint.resume(ctx2, ck, order, scheme, elementary)
"""
from __future__ import annotations

import hashlib

import numpy as np

from . import DSO_TRIPLE_JUMP, DSO_VTV, dso_scheme_coefficients


def scheme_digest(order: int, scheme: int = DSO_TRIPLE_JUMP, elementary: int = DSO_VTV) -> str:
    """SHA-256 (hex) of the pruned coefficients, index arrays and elementary method."""
    a, b, ia, ib, nau, nbu = dso_scheme_coefficients(order, scheme)
    h = hashlib.sha256()
    for arr in (np.asarray(a, np.float64), np.asarray(b, np.float64), np.asarray(ia, np.int64),
                np.asarray(ib, np.int64), np.array([elementary, nau, nbu], np.int64)):
        h.update(arr.tobytes())
    return h.hexdigest()


def capture(ctx, order: int, scheme: int, elementary: int, steps_done: int, dt: float) -> dict:
    return {"psi": ctx.psi(), "steps_done": int(steps_done), "dt": float(dt),
            "digest": scheme_digest(order, scheme, elementary)}


def save(path: str, ck: dict) -> None:
    np.savez(path, psi=ck["psi"], steps_done=ck["steps_done"], dt=ck["dt"], digest=ck["digest"])


def load(path: str) -> dict:
    with np.load(path) as z:
        return {"psi": z["psi"], "steps_done": int(z["steps_done"]), "dt": float(z["dt"]),
                "digest": str(z["digest"])}


def resume(ctx, ck: dict, order: int, scheme: int, elementary: int) -> None:
    """Load the checkpointed psi into `ctx` (already holding the same problem
    and scheme); raises ValueError if the composition differs."""
    if ck["digest"] != scheme_digest(order, scheme, elementary):
        raise ValueError("checkpoint was made with another composition scheme")
    ctx.set_psi(ck["psi"])
