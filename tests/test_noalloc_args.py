"""Argument checks of the Python wrapper of the allocation-free observables
entry point.  The C entry point receives no buffer sizes, so the wrapper must
refuse wrong element types and short buffers before anything is launched;
these checks run on CPU tensors (they come before the device check)."""
import pytest

torch = pytest.importorskip("torch")

import paper_1903_04946_gb300 as dso  # noqa: E402


S, P = 3, 64


def _args():
    psi = torch.zeros(S * P, dtype=torch.complex128)
    V = torch.zeros(S * (S + 1) // 2 * P, dtype=torch.float64)
    out = torch.zeros(S + 1, dtype=torch.float64)
    return psi, V, out


@pytest.mark.parametrize("bad,msg", [
    ("psi_dtype", "psi must be complex128"), ("psi_short", "psi holds"), ("out_dtype", "out must be float64"),
    ("out_short", "out holds"), ("V_dtype", "V must be float64"), ("V_short", "V holds"),
    ("host", "device tensors"), ("numpy", "torch tensors")])
def test_bad_arguments_raise_before_launch(bad, msg):
    psi, V, out = _args()
    if bad == "psi_dtype":
        psi = psi.to(torch.complex64)
    elif bad == "psi_short":
        psi = psi[: S * P - 1]
    elif bad == "out_dtype":
        out = out.to(torch.float32)
    elif bad == "out_short":
        out = out[:S]
    elif bad == "V_dtype":
        V = V.to(torch.float32)
    elif bad == "V_short":
        V = V[:-1]
    elif bad == "numpy":
        psi = psi.numpy()
    with pytest.raises((ValueError, TypeError), match=msg):
        dso.dso_position_observables_noalloc(psi, V, S, P, 0.1, out)
