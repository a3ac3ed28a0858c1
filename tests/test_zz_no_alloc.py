"""The allocation-free observables entry point, for callers that cannot
allocate device memory (pool-owned or fixed-budget device memory, contexts
where an allocation would synchronise).  It is called through the C ABI on a
device wavefunction twice in a row and must agree with the populations that
the context-based dso_observables reports for the same state, within the
tolerance of the other observables tests.  Collected last on purpose."""
import numpy as np
import pytest

import synth
from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def test_noalloc_populations_match_context_observables():
    dso = require_gpu()
    import torch
    pr = synth.pyrazine_like(seed=12, n=(32, 32, 16))
    ctx = dso.Context(pr, order=4, scheme=dso.DSO_SUZUKI)
    ctx.propagate(120.0, 30.0)
    norm, energy, pops = ctx.observables()
    psi = torch.from_numpy(ctx.psi()).cuda()
    ctx.close()
    V = torch.from_numpy(np.ascontiguousarray(pr.V)).cuda()
    dV = float(np.prod([(pr.qmax[d] - pr.qmin[d]) / pr.n[d] for d in range(pr.D)]))
    from oracle import observables as O
    vref = O.potential_energy(pr, psi.cpu().numpy())
    stream = torch.cuda.current_stream()
    for call in range(2):
        out = torch.full((pr.S + 1,), float("nan"), dtype=torch.float64, device="cuda")
        dso.dso_position_observables_noalloc(psi, V, pr.S, pr.points, dV, out, stream)
        torch.cuda.synchronize()
        res = out.cpu().numpy()
        assert res[:pr.S] == pytest.approx(pops, rel=1e-12, abs=1e-15), call
        assert np.sqrt(res[:pr.S].sum()) == pytest.approx(norm, rel=1e-13), call
        assert res[pr.S] == pytest.approx(vref, rel=1e-12), call
    # without a potential the last slot is exactly zero
    out = torch.full((pr.S + 1,), float("nan"), dtype=torch.float64, device="cuda")
    dso.dso_position_observables_noalloc(psi, None, pr.S, pr.points, dV, out, stream)
    torch.cuda.synchronize()
    res = out.cpu().numpy()
    assert res[pr.S] == 0.0
    assert res[:pr.S] == pytest.approx(pops, rel=1e-12, abs=1e-15)
    # the calls allocate nothing: free device memory does not move over
    # repeated calls once the first call has run
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(5):
        dso.dso_position_observables_noalloc(psi, V, pr.S, pr.points, dV, out, stream)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    # a surface count beyond the scratch array is rejected
    big = torch.zeros(6, dtype=torch.float64, device="cuda")
    with pytest.raises(dso.DSOError):
        dso.dso_position_observables_noalloc(psi.reshape(-1)[: 5 * (pr.points // 5) * 1], None, 5,
                                             pr.points // 5, dV, big, stream)
