"""Full-size parity of the benchmarked configuration.

The timed workload is the 3-D three-surface pyrazine-like model on a 64^3
grid per surface, complex128, Suzuki order 6 (25 substeps per step),
dt = 2000/128 a.u., built by the benchmark's own workload function.  Three
time steps exercise every pass kind of the timed run: the first step's
[V F0], the merged step boundary (one potential action with coefficient
a~_last + a~_0), the CUDA-graph replay of the middle steps and the final
[I0 V].  The GPU result is compared with the FP64 oracle element by element
(relative L2 <= 1e-12 and every element within 1e-11 of the largest
amplitude) in four launch configurations:

* the product path with the autotuned kernel plan, on a caller stream as in
  the benchmark (one propagate call of three steps: graph replay);
* the benchmark's timed call pattern (one propagate call per step, whose
  step boundaries are the two actions of the unmerged form);
* the autotuned plan forced through DSO_PLAN (the configuration a profiler
  run reproduces);
* every kernel variant forced on all pass kinds.

The results of the configurations that run the same arithmetic must agree
bitwise; the per-step calls agree bitwise with one call whose boundary is
unmerged (dso_set_boundary_merge(ctx, 0)) and to round-off with the merged
one.
"""
import os

import numpy as np
import pytest

from gpu_util import assert_parity, require_gpu

pytestmark = pytest.mark.gpu

NSTEPS = 3
setup_cache = {}  # results shared between the tests of this module (run in order)


@pytest.fixture(scope="module")
def setup():
    dso = require_gpu()
    import bench
    bench.select_workload("pyrazine64")
    pr = bench.workload(bench.SEED)
    assert tuple(pr.n) == (64, 64, 64) and pr.S == 3
    assert bench.ORDER == 6 and bench.SCHEME_NAME == "suzuki"
    from oracle import propagate as P
    ref = P.propagate(pr, NSTEPS * bench.DT, bench.DT, order=6, scheme="suzuki")
    return dso, bench, pr, ref


def _bench_context(dso, bench, pr, stream):
    ctx = dso.Context(device=0, stream=stream)
    ctx.load_problem(pr)
    dso.dso_set_scheme(ctx.ctx, bench.ORDER, bench.scheme_code())
    return ctx


def test_autotuned_graph_replay(setup, monkeypatch):
    dso, bench, pr, ref = setup
    import torch
    monkeypatch.delenv("DSO_PLAN", raising=False)
    monkeypatch.delenv("DSO_VARIANT", raising=False)
    stream = torch.cuda.Stream()
    ctx = _bench_context(dso, bench, pr, stream)
    ctx.propagate(NSTEPS * bench.DT, bench.DT)
    out = ctx.psi()
    plan = dso.dso_tuned_plan(ctx.ctx)
    ctx.close()
    assert_parity(out, ref)
    setup_cache["graph"] = out
    setup_cache["plan"] = plan



def test_bench_call_pattern(setup, monkeypatch):
    dso, bench, pr, ref = setup
    import torch
    monkeypatch.delenv("DSO_PLAN", raising=False)
    monkeypatch.delenv("DSO_VARIANT", raising=False)
    stream = torch.cuda.Stream()
    ctx = _bench_context(dso, bench, pr, stream)
    with torch.cuda.stream(stream):
        for _ in range(NSTEPS):
            ctx.propagate(bench.DT, bench.DT)
    out = ctx.psi()
    ctx.close()
    assert_parity(out, ref)
    whole = _bench_context(dso, bench, pr, stream)
    dso.dso_set_boundary_merge(whole.ctx, 0)
    whole.propagate(NSTEPS * bench.DT, bench.DT)
    unmerged = whole.psi()
    whole.close()
    assert np.array_equal(out, unmerged)
    if "graph" in setup_cache:
        g = setup_cache["graph"]
        assert np.sqrt(np.sum(np.abs(out - g) ** 2) / np.sum(np.abs(g) ** 2)) < 1e-13


def test_forced_tuned_plan(setup, monkeypatch):
    dso, bench, pr, ref = setup
    import torch
    plan = setup_cache.get("plan")
    if plan is None:
        pytest.skip("needs the autotuned run")
    monkeypatch.setenv("DSO_PLAN", plan)
    stream = torch.cuda.Stream()
    ctx = _bench_context(dso, bench, pr, stream)
    ctx.propagate(NSTEPS * bench.DT, bench.DT)
    out = ctx.psi()
    assert dso.dso_tuned_plan(ctx.ctx) == plan
    ctx.close()
    assert_parity(out, ref)
    assert np.array_equal(out, setup_cache["graph"])


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4])
def test_every_variant_full_size(setup, monkeypatch, variant):
    dso, bench, pr, ref = setup
    import torch
    # the same variant on every pass kind that supports it (4 lines per tile,
    # 16 for the register-resident variant, 2 resident CTAs per SM for the
    # persistent TMA variant)
    entries = []
    for axis in range(3):
        for staged in (0, 1):
            g = 16 if variant == 4 else 4
            entries.append(f"{axis},{staged},{variant},{g},{2 if variant == 3 else 0};")
    monkeypatch.setenv("DSO_PLAN", "".join(entries))
    stream = torch.cuda.Stream()
    ctx = _bench_context(dso, bench, pr, stream)
    ctx.propagate(NSTEPS * bench.DT, bench.DT)
    out = ctx.psi()
    got_plan = dso.dso_tuned_plan(ctx.ctx)
    ctx.close()
    assert_parity(out, ref)
    if "graph" in setup_cache:
        assert np.array_equal(out, setup_cache["graph"]), got_plan
