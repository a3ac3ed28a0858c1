"""Checkpoint / resume: the composition digest (host only) and an exact
resume on the GPU."""
import numpy as np
import pytest

import synth
from gpu_util import require_gpu
import paper_1903_04946_gb300 as dso
from paper_1903_04946_gb300 import checkpoint


def test_digest_names_the_composition():
    dso.build()   # host-only entry point of the library (no GPU needed)
    dso.load()
    d = checkpoint.scheme_digest(6, dso.DSO_SUZUKI, dso.DSO_VTV)
    assert d == checkpoint.scheme_digest(6, dso.DSO_SUZUKI, dso.DSO_VTV)
    others = {checkpoint.scheme_digest(6, dso.DSO_TRIPLE_JUMP, dso.DSO_VTV),
              checkpoint.scheme_digest(4, dso.DSO_SUZUKI, dso.DSO_VTV),
              checkpoint.scheme_digest(6, dso.DSO_SUZUKI, dso.DSO_TVT)}
    assert d not in others and len(others) == 3


@pytest.mark.gpu
@pytest.mark.parametrize("el,merged", [("VTV", 0), ("VTV", 1), ("TVT", 1)])
def test_resume_is_exact(tmp_path, el, merged):
    """Bitwise with the unmerged VTV boundary; to round-off where the whole
    run merges the boundary actions (or, in TVT, keeps them in one pass)."""
    require_gpu()
    code = dso.DSO_TVT if el == "TVT" else dso.DSO_VTV
    pr = synth.pyrazine_like(seed=41, n=(16, 32, 16))
    dt = 25.0
    whole = dso.Context(pr, order=6, scheme=dso.DSO_SUZUKI, elementary=code)
    dso.dso_set_boundary_merge(whole.ctx, merged)
    whole.propagate(6 * dt, dt)
    ref = whole.psi()
    whole.close()

    first = dso.Context(pr, order=6, scheme=dso.DSO_SUZUKI, elementary=code)
    dso.dso_set_boundary_merge(first.ctx, merged)
    first.propagate(2 * dt, dt)
    first.propagate(dt, dt)                     # chunks of any size
    ck = checkpoint.capture(first, 6, dso.DSO_SUZUKI, code, 3, dt)
    first.close()
    checkpoint.save(str(tmp_path / "ck.npz"), ck)

    ck2 = checkpoint.load(str(tmp_path / "ck.npz"))
    assert ck2["steps_done"] == 3 and ck2["dt"] == dt
    second = dso.Context(pr, order=6, scheme=dso.DSO_SUZUKI, elementary=code)
    dso.dso_set_boundary_merge(second.ctx, merged)
    with pytest.raises(ValueError):
        checkpoint.resume(second, ck2, 4, dso.DSO_SUZUKI, code)
    checkpoint.resume(second, ck2, 6, dso.DSO_SUZUKI, code)
    second.propagate(3 * dt, dt)
    out = second.psi()
    second.close()
    if el == "VTV" and not merged:
        assert np.array_equal(out, ref)
    else:  # one merged action against two, or an extra FFT round trip between them
        assert np.sqrt(np.sum(np.abs(out - ref) ** 2) / np.sum(np.abs(ref) ** 2)) < 1e-13
