"""CPU-side checks of the CUDA library: it builds for sm_103a, loads, exports
every entry point declared in include/dso.h, and its host-only coefficient
code reproduces Table II and the oracle's coefficients.  No GPU needed."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1903_04946_gb300 as dso
from oracle import coefficients as C

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    dso.build()
    return dso.load()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(dso_\w+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert declared, "no declarations found"
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(dso.EXPORTS) | (declared - set(dso.EXPORTS))
    assert set(dso.EXPORTS) <= declared


def test_library_targets_sm103a():
    out = os.popen(f"/usr/local/cuda/bin/cuobjdump --list-elf {dso.LIB} 2>/dev/null").read()
    if not out:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in out


def _table2():
    rows = []
    for line in open(os.path.join(ROOT, "tests", "golden", "table2.txt")):
        if line.startswith("#") or not line.strip():
            continue
        sch, o, before, after, na, nb = line.split()
        rows.append((sch, int(o), int(after), int(na), int(nb)))
    return rows


@pytest.mark.parametrize("row", _table2(), ids=lambda r: f"{r[0]}{r[1]}")
def test_library_coefficients_match_table2(lib, row):
    sch, order, after, na, nb = row
    scheme = dso.SCHEME_CODES.get(sch, dso.DSO_TRIPLE_JUMP)
    a, b, ia, ib, nau, nbu = dso.dso_scheme_coefficients(order, scheme)
    assert len(a) + len(b) == after
    assert (nau, nbu) == (na, nb)
    assert len(a) == len(b) + 1


@pytest.mark.parametrize("scheme", [dso.DSO_TRIPLE_JUMP, dso.DSO_SUZUKI])
@pytest.mark.parametrize("order", [2, 4, 6, 8, 10])
def test_library_coefficients_match_oracle(lib, scheme, order):
    a, b, ia, ib, nau, nbu = dso.dso_scheme_coefficients(order, scheme)
    sp = C.Splitting(order, C.SUZUKI if scheme == dso.DSO_SUZUKI else C.TRIPLE_JUMP)
    assert np.max(np.abs(a - np.array(sp.a))) <= 2e-16 * np.max(np.abs(a))
    assert np.max(np.abs(b - np.array(sp.b))) <= 2e-16 * np.max(np.abs(b))
    assert list(ia) == list(sp.Ia) and list(ib) == list(sp.Ib)


def test_library_first_order_coefficients(lib):
    """Order 1 is the first-order VT / TV algorithm (Sec. II E): one action of
    each operator with unit coefficient, written as a = (1, 0), b = (1) so
    that the composed-step machinery runs it (the trailing action is the
    zero-time identity)."""
    a, b, ia, ib, nau, nbu = dso.dso_scheme_coefficients(1, dso.DSO_TRIPLE_JUMP)
    assert list(a) == [1.0, 0.0] and list(b) == [1.0]
    assert list(ia) == [0, 1] and list(ib) == [0] and (nau, nbu) == (2, 1)
    oa, ob = C.first_order()
    assert list(b) == ob and a[0] == oa[0]


def test_library_rejects_bad_scheme(lib):
    with pytest.raises(dso.DSOError):
        dso.dso_scheme_coefficients(3, dso.DSO_TRIPLE_JUMP)
    with pytest.raises(dso.DSOError):
        dso.dso_scheme_coefficients(4, 7)
    assert "scheme" in dso.dso_last_error() or "order" in dso.dso_last_error()


def test_create_without_gpu_fails_cleanly(lib):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    ctx = ctypes.c_void_p()
    st = lib.dso_create(ctypes.byref(ctx), 0, dso.DSO_FP64, None)
    assert st != dso.DSO_OK
    assert not ctx.value


# a symmetric 7-stage composition that is not one of the recursive schemes
CUSTOM7 = [0.21, -0.13, 0.37, 0.1, 0.37, -0.13, 0.21]


def test_composition_coefficients_from_gammas(lib):
    """dso_composition_coefficients expands any symmetric composition as the
    built-in schemes are expanded: the triple-jump gammas give the order-4
    triple-jump coefficients, and a custom composition matches the oracle's
    expansion of the same gammas."""
    x = 1.0 / (2.0 - 2.0 ** (1.0 / 3.0))
    a, b, ia, ib, nau, nbu = dso.dso_composition_coefficients([x, 1.0 - 2.0 * x, x])
    ra, rb, ria, rib, rnau, rnbu = dso.dso_scheme_coefficients(4, dso.DSO_TRIPLE_JUMP)
    assert np.max(np.abs(a - ra)) < 1e-15 and np.max(np.abs(b - rb)) < 1e-15
    assert list(ia) == list(ria) and list(ib) == list(rib) and (nau, nbu) == (rnau, rnbu)
    g = np.array(CUSTOM7)
    g[3] = 1.0 - (g.sum() - g[3])                      # sum exactly 1
    a, b, ia, ib, nau, nbu = dso.dso_composition_coefficients(g)
    sp = C.Splitting(0, C.TRIPLE_JUMP, gammas=g)
    assert np.max(np.abs(a - np.array(sp.a))) <= 2e-16 and np.max(np.abs(b - np.array(sp.b))) <= 2e-16
    assert list(ia) == list(sp.Ia) and list(ib) == list(sp.Ib)


@pytest.mark.parametrize("bad", [[0.5, 0.6], [0.4, 0.2, 0.3], [0.5, 0.0, 0.5], [float("nan")], []])
def test_composition_rejects_bad_gammas(lib, bad):
    with pytest.raises(dso.DSOError):
        dso.dso_composition_coefficients(bad)


@pytest.mark.parametrize("order", [6, 8])
def test_library_optimal_coefficients_match_oracle(lib, order):
    a, b, ia, ib, nau, nbu = dso.dso_scheme_coefficients(order, dso.DSO_OPTIMAL)
    sp = C.Splitting(order, C.OPTIMAL)
    assert np.allclose(a, sp.a, rtol=0, atol=1e-15) and np.allclose(b, sp.b, rtol=0, atol=1e-15)
    assert list(ia) == sp.Ia and list(ib) == sp.Ib
    with pytest.raises(dso.DSOError):
        dso.dso_scheme_coefficients(4, dso.DSO_OPTIMAL)


@pytest.mark.parametrize("name,arg", [("dso_set_plane_pass", 1), ("dso_set_kinetic_mode", 1),
                                      ("dso_set_operator_mode", 1), ("dso_set_boundary_merge", 1)])
def test_mode_setters_reject_a_null_context(lib, name, arg):
    """The mode setters check their context before touching a device."""
    assert getattr(lib, name)(None, arg) == dso.DSO_EINVAL
