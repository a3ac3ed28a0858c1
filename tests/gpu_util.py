"""Helpers for the GPU parity tests (CUDA library vs the CPU oracle)."""
import numpy as np
import pytest

TOL = 1e-12  # relative L2, FP64 (spec parity bound)


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1903_04946_gb300 as dso
    dso.build()
    dso.load()
    return dso


def gpu_propagate(problem, order, scheme, t, dt, psi=None, elementary="VTV", fp32=False):
    import paper_1903_04946_gb300 as dso
    sch = dso.SCHEME_CODES[scheme]
    el = {"VTV": dso.DSO_VTV, "TVT": dso.DSO_TVT, "VT": dso.DSO_VT, "TV": dso.DSO_TV}[elementary]
    ctx = dso.Context(problem, order=order, scheme=sch, elementary=el,
                      precision=dso.DSO_FP32 if fp32 else dso.DSO_FP64)
    try:
        if psi is not None:
            ctx.set_psi(psi)
        ctx.propagate(t, dt)
        return ctx.psi()
    finally:
        ctx.close()


def oracle_propagate(problem, order, scheme, t, dt, psi=None, elementary="VTV"):
    from oracle import propagate as P
    return P.propagate(problem, t, dt, order=order, scheme=scheme, psi=psi, elementary=elementary)


def rel_l2(a, b):
    return float(np.sqrt(np.sum(np.abs(a - b) ** 2) / np.sum(np.abs(b) ** 2)))


def assert_parity(gpu, ref, tol=TOL):
    assert gpu.shape == ref.shape
    assert np.all(np.isfinite(gpu))
    err = rel_l2(gpu, ref)
    # element by element: no entry may differ by more than tol x the largest amplitude
    emax = float(np.max(np.abs(gpu - ref)) / np.max(np.abs(ref)))
    assert err <= tol and emax <= 10 * tol, (err, emax)
    return err
