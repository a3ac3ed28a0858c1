"""Python binding of the GB300 diabatic split-operator library (include/dso.h).

Argument marshalling only: every function here forwards to the C entry point
of the same name in ``libdso_gb300.so``; all propagation work runs in the
library's CUDA kernels.  Host arrays are numpy (or CPU torch) arrays, device
arrays are CUDA torch tensors; streams are torch CUDA streams (or raw
cudaStream_t integers).  There is no CPU fallback: if the library is missing
or cannot be loaded, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB, build  # noqa: F401

DSO_OK, DSO_EINVAL, DSO_ENOMEM, DSO_ECUDA, DSO_ESTATE, DSO_ETIMEOUT, DSO_ENUMERIC = 0, -1, -2, -3, -4, -5, -6
DSO_HOST, DSO_DEVICE = 0, 1
DSO_FP64, DSO_FP32 = 0, 1
DSO_TRIPLE_JUMP, DSO_SUZUKI, DSO_OPTIMAL = 0, 1, 2
SCHEME_CODES = {"triple_jump": DSO_TRIPLE_JUMP, "suzuki": DSO_SUZUKI, "optimal": DSO_OPTIMAL}
DSO_VTV, DSO_TVT, DSO_VT, DSO_TV = 0, 1, 2, 3
DSO_KINETIC_AUTO, DSO_KINETIC_JOINT, DSO_KINETIC_AXES = -1, 0, 1
DSO_PLANE_AUTO, DSO_PLANE_OFF, DSO_PLANE_ON = -1, 0, 1
DSO_OPERATORS_AUTO, DSO_OPERATORS_TABLES, DSO_OPERATORS_ON_THE_FLY = -1, 0, 1

EXPORTS = (
    "dso_create", "dso_destroy", "dso_set_grid", "dso_set_batch", "dso_set_masses", "dso_load_potential",
    "dso_set_scheme", "dso_set_psi", "dso_propagate", "dso_get_psi", "dso_observables",
    "dso_scheme_coefficients", "dso_profile_steps", "dso_launch_count", "dso_last_error",
    "dso_position_observables_noalloc", "dso_busy", "dso_tuned_plan", "dso_set_composition",
    "dso_composition_coefficients", "dso_set_norm_check", "dso_fp64_issue_rate", "dso_inner",
    "dso_phase_at_density_maximum", "dso_set_wait_probe", "dso_psi_device_pointer", "dso_set_pass_limits",
    "dso_batch_create", "dso_batch_destroy", "dso_batch_add", "dso_batch_step", "dso_batch_sync",
    "dso_batch_slot_status", "dso_batch_retire", "dso_batch_launch_count", "dso_batch_busy",
    "dso_set_kinetic_mode", "dso_set_boundary_merge", "dso_set_plane_pass", "dso_set_operator_mode",
    "dso_operators_on_the_fly",
)

_lib = None


class DSOError(RuntimeError):
    def __init__(self, status, where):
        msg = _lib.dso_last_error().decode() if _lib is not None else "library not loaded"
        super().__init__(f"{where} failed with status {status}: {msg}")
        self.status = status


def load(path: str = LIB):
    """Load the shared library (it must have been built with ``build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing: run paper_1903_04946_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    pd, pi = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    sig = {
        "dso_create": (i32, [ctypes.POINTER(vp), i32, i32, vp]),
        "dso_destroy": (None, [vp]),
        "dso_set_grid": (i32, [vp, i32, ctypes.POINTER(i64), pd, pd]),
        "dso_set_masses": (i32, [vp, pd]),
        "dso_set_batch": (i32, [vp, i32]),
        "dso_load_potential": (i32, [vp, i32, vp, i32]),
        "dso_set_scheme": (i32, [vp, i32, i32, i32, i32]),
        "dso_set_psi": (i32, [vp, vp, i32]),
        "dso_propagate": (i32, [vp, dbl, dbl]),
        "dso_get_psi": (i32, [vp, vp, i32]),
        "dso_observables": (i32, [vp, pd, pd, pd]),
        "dso_scheme_coefficients": (i32, [i32, i32, pi, pi, pd, pd, pi, pi, pi, pi]),
        "dso_profile_steps": (i32, [vp, dbl, i32, i32, pi, pi, pi, pi, pi, pd, pi, pi]),
        "dso_launch_count": (i64, [vp]),
        "dso_busy": (i32, [vp]),
        "dso_tuned_plan": (i32, [vp, ctypes.c_char_p, i32]),
        "dso_set_composition": (i32, [vp, i32, pd, i32]),
        "dso_set_norm_check": (i32, [vp, dbl]),
        "dso_composition_coefficients": (i32, [i32, pd, pi, pi, pd, pd, pi, pi, pi, pi]),
        "dso_last_error": (ctypes.c_char_p, []),
        "dso_position_observables_noalloc": (i32, [vp, vp, i32, i64, dbl, vp, vp]),
        "dso_fp64_issue_rate": (i32, [i32, pd]),
        "dso_inner": (i32, [vp, vp, i32, pd, pd]),
        "dso_phase_at_density_maximum": (i32, [vp, ctypes.POINTER(i64), pd]),
        "dso_set_wait_probe": (i32, [vp, i32]),
        "dso_psi_device_pointer": (i32, [vp, ctypes.POINTER(vp)]),
        "dso_set_pass_limits": (i32, [vp, i32, i32]),
        "dso_set_kinetic_mode": (i32, [vp, i32]),
        "dso_set_boundary_merge": (i32, [vp, i32]),
        "dso_set_plane_pass": (i32, [vp, i32]),
        "dso_set_operator_mode": (i32, [vp, i32]),
        "dso_operators_on_the_fly": (i32, [vp]),
        "dso_batch_create": (i32, [ctypes.POINTER(vp), i32, i32, vp]),
        "dso_batch_destroy": (None, [vp]),
        "dso_batch_add": (i32, [vp, vp, dbl, dbl, ctypes.POINTER(i32)]),
        "dso_batch_step": (i32, [vp, ctypes.POINTER(i32)]),
        "dso_batch_sync": (i32, [vp]),
        "dso_batch_slot_status": (i32, [vp, i32, ctypes.POINTER(i64), ctypes.POINTER(i64)]),
        "dso_batch_retire": (i32, [vp, i32]),
        "dso_batch_launch_count": (i64, [vp]),
        "dso_batch_busy": (i32, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(status, where):
    if status != DSO_OK:
        raise DSOError(status, where)


def _ptr(buf, writable=False):
    """(pointer, where) of a numpy array or torch tensor (C-contiguous)."""
    try:
        import torch
        if isinstance(buf, torch.Tensor):
            if not buf.is_contiguous():
                raise ValueError("tensor must be contiguous")
            return ctypes.c_void_p(buf.data_ptr()), (DSO_DEVICE if buf.is_cuda else DSO_HOST)
    except ImportError:  # pragma: no cover
        pass
    arr = np.asarray(buf)
    if not arr.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    if writable and not arr.flags["WRITEABLE"]:
        raise ValueError("array must be writeable")
    return ctypes.c_void_p(arr.ctypes.data), DSO_HOST


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


# --- entry points, same names as include/dso.h -----------------------------

def dso_create(device: int = 0, precision: int = DSO_FP64, stream=None):
    lib = load()
    ctx = ctypes.c_void_p()
    _check(lib.dso_create(ctypes.byref(ctx), device, precision, _stream_handle(stream)), "dso_create")
    return ctx


def dso_destroy(ctx):
    load().dso_destroy(ctx)


def dso_set_grid(ctx, n, qmin, qmax):
    D = len(n)
    _check(load().dso_set_grid(ctx, D, (ctypes.c_int64 * D)(*[int(x) for x in n]),
                               (ctypes.c_double * D)(*[float(x) for x in qmin]),
                               (ctypes.c_double * D)(*[float(x) for x in qmax])), "dso_set_grid")


def dso_set_batch(ctx, B):
    _check(load().dso_set_batch(ctx, int(B)), "dso_set_batch")


def dso_set_masses(ctx, m):
    D = len(m)
    _check(load().dso_set_masses(ctx, (ctypes.c_double * D)(*[float(x) for x in m])), "dso_set_masses")


def dso_load_potential(ctx, S, V):
    if isinstance(V, np.ndarray):
        V = np.ascontiguousarray(V, dtype=np.float64)
    p, where = _ptr(V)
    _check(load().dso_load_potential(ctx, int(S), p, where), "dso_load_potential")


def dso_set_scheme(ctx, order, scheme=DSO_TRIPLE_JUMP, elementary=DSO_VTV, prune=1):
    _check(load().dso_set_scheme(ctx, order, scheme, elementary, prune), "dso_set_scheme")


def dso_set_psi(ctx, psi):
    """psi must have the context's element type (complex128 for DSO_FP64,
    complex64 for DSO_FP32)."""
    if isinstance(psi, np.ndarray):
        if psi.dtype not in (np.complex64, np.complex128):
            psi = psi.astype(np.complex128)
        psi = np.ascontiguousarray(psi)
    p, where = _ptr(psi)
    _check(load().dso_set_psi(ctx, p, where), "dso_set_psi")


def dso_propagate(ctx, t, dt):
    _check(load().dso_propagate(ctx, float(t), float(dt)), "dso_propagate")


def dso_get_psi(ctx, out):
    p, where = _ptr(out, writable=True)
    _check(load().dso_get_psi(ctx, p, where), "dso_get_psi")
    return out


def dso_observables(ctx, S, B=1):
    """(norm, energy, pops); with B > 1 jobs, arrays of B, B and (B, S)."""
    norm, energy = (ctypes.c_double * B)(), (ctypes.c_double * B)()
    pops = (ctypes.c_double * (B * S))()
    _check(load().dso_observables(ctx, norm, energy, pops), "dso_observables")
    if B == 1:
        return norm[0], energy[0], np.array(pops[:], dtype=np.float64)
    return (np.array(norm[:]), np.array(energy[:]), np.array(pops[:], dtype=np.float64).reshape(B, S))


def dso_inner(ctx, phi, B=1):
    """<psi|phi> of the context's psi with phi (same layout and precision),
    one complex number per job (a scalar when B == 1)."""
    if isinstance(phi, np.ndarray):
        phi = np.ascontiguousarray(phi)
    p, where = _ptr(phi)
    re, im = (ctypes.c_double * B)(), (ctypes.c_double * B)()
    _check(load().dso_inner(ctx, p, where, re, im), "dso_inner")
    out = np.array(re[:]) + 1j * np.array(im[:])
    return complex(out[0]) if B == 1 else out


def dso_phase_at_density_maximum(ctx, S, B=1):
    """(flat indices, phases) of every job's surfaces at their density
    maxima, arrays of B*S entries (job-major)."""
    idx, ph = (ctypes.c_int64 * (B * S))(), (ctypes.c_double * (B * S))()
    _check(load().dso_phase_at_density_maximum(ctx, idx, ph), "dso_phase_at_density_maximum")
    return np.array(idx[:], dtype=np.int64), np.array(ph[:])


def dso_scheme_coefficients(order, scheme=DSO_TRIPLE_JUMP):
    """(a~, b~, I^a, I^b, N_a^unq, N_b^unq) of a composed scheme (host only)."""
    lib = load()
    na, nb, nau, nbu = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib.dso_scheme_coefficients(order, scheme, ctypes.byref(na), ctypes.byref(nb), None, None, None, None,
                                       ctypes.byref(nau), ctypes.byref(nbu)), "dso_scheme_coefficients")
    a = (ctypes.c_double * na.value)()
    b = (ctypes.c_double * nb.value)()
    ia = (ctypes.c_int * na.value)()
    ib = (ctypes.c_int * nb.value)()
    _check(lib.dso_scheme_coefficients(order, scheme, None, None, a, b, ia, ib, None, None),
           "dso_scheme_coefficients")
    return (np.array(a[:]), np.array(b[:]), np.array(ia[:]), np.array(ib[:]), nau.value, nbu.value)


def dso_profile_steps(ctx, dt, nsteps, max_kinds=16):
    """Per kind of pass: dicts with axis, flags, surfaces, launches_per_step,
    avg_ms (CUDA events around every launch on the context's stream)."""
    lib = load()
    nk = ctypes.c_int()
    ax, fl, sv, cnt, gl, var = [(ctypes.c_int * max_kinds)() for _ in range(6)]
    ms = (ctypes.c_double * max_kinds)()
    _check(lib.dso_profile_steps(ctx, float(dt), int(nsteps), max_kinds, ctypes.byref(nk), ax, fl, sv, cnt, ms,
                                 gl, var), "dso_profile_steps")
    return [dict(axis=ax[k], flags=fl[k], surfaces=sv[k], launches_per_step=cnt[k], avg_ms=ms[k],
                 tile_lines=gl[k], variant=var[k]) for k in range(min(nk.value, max_kinds))]


def dso_busy(ctx) -> bool:
    r = load().dso_busy(ctx)
    if r < 0:
        raise DSOError(r, "dso_busy")
    return r == 1


def dso_set_composition(ctx, gammas, elementary=DSO_VTV):
    """Use the symmetric composition with elementary coefficients `gammas`."""
    g = np.ascontiguousarray(gammas, dtype=np.float64)
    _check(load().dso_set_composition(ctx, int(g.size), g.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      elementary), "dso_set_composition")


def dso_set_norm_check(ctx, tol):
    """Fail dso_propagate (DSO_ENUMERIC) when a job's norm drifts by more
    than `tol` relative; 0 switches the check off."""
    _check(load().dso_set_norm_check(ctx, float(tol)), "dso_set_norm_check")


def dso_composition_coefficients(gammas):
    """(a~, b~, I^a, I^b, N_a^unq, N_b^unq) of a user composition (host only)."""
    lib = load()
    g = np.ascontiguousarray(gammas, dtype=np.float64)
    gp = g.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    na, nb, nau, nbu = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib.dso_composition_coefficients(int(g.size), gp, ctypes.byref(na), ctypes.byref(nb), None, None, None,
                                            None, ctypes.byref(nau), ctypes.byref(nbu)),
           "dso_composition_coefficients")
    a = (ctypes.c_double * na.value)()
    b = (ctypes.c_double * nb.value)()
    ia = (ctypes.c_int * na.value)()
    ib = (ctypes.c_int * nb.value)()
    _check(lib.dso_composition_coefficients(int(g.size), gp, None, None, a, b, ia, ib, None, None),
           "dso_composition_coefficients")
    return (np.array(a[:]), np.array(b[:]), np.array(ia[:]), np.array(ib[:]), nau.value, nbu.value)


def dso_set_wait_probe(ctx, polls):
    """Diagnostics: a bounded wait in the TMA variant that must give up."""
    _check(load().dso_set_wait_probe(ctx, int(polls)), "dso_set_wait_probe")


def dso_psi_device_pointer(ctx) -> int:
    """Device address of the context's psi (borrowed; see include/dso.h)."""
    p = ctypes.c_void_p()
    _check(load().dso_psi_device_pointer(ctx, ctypes.byref(p)), "dso_psi_device_pointer")
    return int(p.value)


def device_view(ptr: int, shape, dtype, device=0):
    """A torch tensor that views `shape` elements of `dtype` at device address
    `ptr` without a copy (through __cuda_array_interface__); the memory stays
    owned by whoever allocated it."""
    import torch
    typestr = {np.dtype(np.complex128): "<c16", np.dtype(np.complex64): "<c8",
               np.dtype(np.float64): "<f8"}[np.dtype(dtype)]

    class _View:
        __cuda_array_interface__ = {"shape": tuple(int(x) for x in shape), "typestr": typestr,
                                    "data": (int(ptr), False), "version": 3, "strides": None}
    return torch.as_tensor(_View(), device=f"cuda:{device}")


def dso_set_pass_limits(ctx, max_line, max_tile):
    _check(load().dso_set_pass_limits(ctx, int(max_line), int(max_tile)), "dso_set_pass_limits")


def dso_set_kinetic_mode(ctx, mode):
    _check(load().dso_set_kinetic_mode(ctx, int(mode)), "dso_set_kinetic_mode")


def dso_set_boundary_merge(ctx, merged):
    _check(load().dso_set_boundary_merge(ctx, int(merged)), "dso_set_boundary_merge")


def dso_set_plane_pass(ctx, mode):
    _check(load().dso_set_plane_pass(ctx, int(mode)), "dso_set_plane_pass")


def dso_set_operator_mode(ctx, mode):
    _check(load().dso_set_operator_mode(ctx, int(mode)), "dso_set_operator_mode")


def dso_operators_on_the_fly(ctx) -> bool:
    r = load().dso_operators_on_the_fly(ctx)
    _check(min(r, 0), "dso_operators_on_the_fly")
    return r == 1


def dso_batch_create(device: int = 0, precision: int = DSO_FP64, stream=None):
    b = ctypes.c_void_p()
    _check(load().dso_batch_create(ctypes.byref(b), device, precision, _stream_handle(stream)), "dso_batch_create")
    return b


def dso_batch_destroy(batch):
    load().dso_batch_destroy(batch)


def dso_batch_add(batch, ctx, t, dt) -> int:
    slot = ctypes.c_int()
    _check(load().dso_batch_add(batch, ctx, float(t), float(dt), ctypes.byref(slot)), "dso_batch_add")
    return slot.value


def dso_batch_step(batch) -> int:
    active = ctypes.c_int()
    _check(load().dso_batch_step(batch, ctypes.byref(active)), "dso_batch_step")
    return active.value


def dso_batch_sync(batch):
    _check(load().dso_batch_sync(batch), "dso_batch_sync")


def dso_batch_slot_status(batch, slot):
    done, total = ctypes.c_int64(), ctypes.c_int64()
    _check(load().dso_batch_slot_status(batch, int(slot), ctypes.byref(done), ctypes.byref(total)),
           "dso_batch_slot_status")
    return done.value, total.value


def dso_batch_retire(batch, slot):
    _check(load().dso_batch_retire(batch, int(slot)), "dso_batch_retire")


def dso_batch_launch_count(batch) -> int:
    return int(load().dso_batch_launch_count(batch))


def dso_batch_busy(batch) -> bool:
    r = load().dso_batch_busy(batch)
    if r < 0:
        raise DSOError(r, "dso_batch_busy")
    return r == 1


class Batch:
    """Batch slots: Context objects join with their own t and dt, advance
    one composed step per launch, and leave when retired."""

    def __init__(self, device: int = 0, precision: int = DSO_FP64, stream=None):
        self.b = dso_batch_create(device, precision, stream)
        self.jobs = {}

    def add(self, ctx: "Context", t, dt) -> int:
        slot = dso_batch_add(self.b, ctx.ctx, t, dt)
        self.jobs[slot] = ctx
        return slot

    def step(self) -> int:
        return dso_batch_step(self.b)

    def run(self):
        """Step until every job has finished."""
        while self.step() > 0:
            pass
        dso_batch_sync(self.b)

    def status(self, slot):
        return dso_batch_slot_status(self.b, slot)

    def busy(self) -> bool:
        return dso_batch_busy(self.b)

    def retire(self, slot) -> "Context":
        dso_batch_retire(self.b, slot)
        return self.jobs.pop(slot)

    def close(self):
        if self.b is not None:
            dso_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dso_tuned_plan(ctx) -> str:
    """The autotuned kernel configuration, in the DSO_PLAN format."""
    buf = ctypes.create_string_buffer(1024)
    r = load().dso_tuned_plan(ctx, buf, 1024)
    if r < 0:
        raise DSOError(r, "dso_tuned_plan")
    return buf.value.decode()


def dso_launch_count(ctx) -> int:
    return int(load().dso_launch_count(ctx))


def dso_position_observables_noalloc(psi, V, S, P, dV, out, stream=None):
    """Allocation-free populations and potential energy of a device psi.
    psi, V (or None) and out are CUDA tensors; out receives S + 1 doubles.
    For callers that cannot allocate device memory; see include/dso.h.

    The C entry point receives no buffer sizes, so the element types and
    counts are checked here, before anything is launched: psi complex128 with
    at least S * P elements, V float64 with at least S(S+1)/2 * P, out float64
    with at least S + 1, all on one GPU (the call runs with that GPU
    current)."""
    import torch
    S, P = int(S), int(P)
    if not isinstance(psi, torch.Tensor) or not isinstance(out, torch.Tensor) or \
            (V is not None and not isinstance(V, torch.Tensor)):
        raise TypeError("psi, V and out must be torch tensors")
    if psi.dtype != torch.complex128:
        raise ValueError("psi must be complex128")
    if out.dtype != torch.float64:
        raise ValueError("out must be float64")
    if S >= 1 and P >= 1:
        if psi.numel() < S * P:
            raise ValueError(f"psi holds {psi.numel()} elements, needs S * P = {S * P}")
        if out.numel() < S + 1:
            raise ValueError(f"out holds {out.numel()} elements, needs S + 1 = {S + 1}")
        if V is not None:
            if V.dtype != torch.float64:
                raise ValueError("V must be float64")
            if V.numel() < S * (S + 1) // 2 * P:
                raise ValueError(f"V holds {V.numel()} elements, needs S(S+1)/2 * P = {S * (S + 1) // 2 * P}")
    tensors = [psi, out] + ([V] if V is not None else [])
    if not all(t.is_cuda for t in tensors):
        raise ValueError("psi, V and out must be device tensors")
    if len({t.device for t in tensors}) != 1:
        raise ValueError("psi, V and out must be on one device")
    pp, _ = _ptr(psi)
    po, _ = _ptr(out, writable=True)
    pv = _ptr(V)[0] if V is not None else None
    with torch.cuda.device(psi.device):
        _check(load().dso_position_observables_noalloc(pp, pv, S, P, float(dV), po, _stream_handle(stream)),
               "dso_position_observables_noalloc")
    return out


def dso_fp64_issue_rate(device: int = 0) -> float:
    """FP64 FMA instructions per second the device retires (microbenchmark)."""
    r = ctypes.c_double()
    _check(load().dso_fp64_issue_rate(int(device), ctypes.byref(r)), "dso_fp64_issue_rate")
    return r.value


def dso_last_error() -> str:
    return load().dso_last_error().decode()


class Context:
    """Owns one dso context; a convenience holder over the functions above."""

    def __init__(self, problem=None, device: int = 0, stream=None, order: int = 2,
                 scheme: int = DSO_TRIPLE_JUMP, elementary: int = DSO_VTV, precision: int = DSO_FP64):
        self.ctx = dso_create(device, precision, stream)
        self.dtype = np.complex64 if precision == DSO_FP32 else np.complex128
        self.S = None
        self.B = 1
        self.shape = None
        if problem is not None:
            self.load_problem(problem)
            dso_set_scheme(self.ctx, order, scheme, elementary)

    def load_problem(self, pr):
        dso_set_grid(self.ctx, pr.n, pr.qmin, pr.qmax)
        dso_set_masses(self.ctx, pr.mass)
        dso_load_potential(self.ctx, pr.S, pr.V)
        dso_set_psi(self.ctx, np.ascontiguousarray(pr.psi0, dtype=self.dtype))
        self.S = pr.S
        self.B = 1
        self.shape = (pr.S,) + tuple(pr.n)

    def load_batch(self, problems):
        """B jobs on one grid (same n, qmin, qmax, masses, S), each with its
        own potential and initial state."""
        p0 = problems[0]
        for pr in problems[1:]:
            if (pr.n, pr.qmin, pr.qmax, pr.mass, pr.S) != (p0.n, p0.qmin, p0.qmax, p0.mass, p0.S):
                raise ValueError("batched jobs must share grid, masses and surface count")
        dso_set_grid(self.ctx, p0.n, p0.qmin, p0.qmax)
        dso_set_batch(self.ctx, len(problems))
        dso_set_masses(self.ctx, p0.mass)
        dso_load_potential(self.ctx, p0.S, np.ascontiguousarray(np.stack([pr.V for pr in problems])))
        dso_set_psi(self.ctx, np.ascontiguousarray(np.stack([pr.psi0 for pr in problems]), dtype=self.dtype))
        self.S = p0.S
        self.B = len(problems)
        self.shape = (self.B, p0.S) + tuple(p0.n)

    def propagate(self, t, dt):
        dso_propagate(self.ctx, t, dt)

    def set_psi(self, psi):
        dso_set_psi(self.ctx, np.ascontiguousarray(psi, dtype=self.dtype))

    def psi(self) -> np.ndarray:
        out = np.empty(self.shape, dtype=self.dtype)
        return dso_get_psi(self.ctx, out)

    def observables(self):
        return dso_observables(self.ctx, self.S, self.B)

    def inner(self, phi):
        """<psi|phi> per job (Sec. II A); omega = -2 Im of it."""
        return dso_inner(self.ctx, np.ascontiguousarray(phi, dtype=self.dtype) if isinstance(phi, np.ndarray)
                         else phi, self.B)

    def phase_at_density_maximum(self):
        return dso_phase_at_density_maximum(self.ctx, self.S, self.B)

    def close(self):
        if self.ctx is not None:
            dso_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
