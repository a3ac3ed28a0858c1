"""Serving loop: jobs of different dimension, surface count, grid and order
arrive while others run, are admitted by device-memory footprint, advance
concurrently on their own streams, and each result equals the job run alone
(relative L2 <= 1e-12, the FP64 parity tolerance; in practice bitwise)."""
import numpy as np
import pytest

from gpu_util import rel_l2, require_gpu

pytestmark = pytest.mark.gpu


def _alone(job):
    import paper_1903_04946_gb300 as dso
    ctx = dso.Context(job.problem, order=job.order, scheme=job.scheme)
    ctx.propagate(job.t, job.dt)
    out = ctx.psi()
    ctx.close()
    return out


def test_served_results_equal_alone():
    require_gpu()
    from paper_1903_04946_gb300 import serving
    jobs = serving.make_jobs(n_jobs=12, seed=77, load=4.0, max_points=1 << 14)
    for j in jobs:   # short runs: cap the steps, keep t a multiple of dt
        j.t = j.dt * min(int(round(j.t / j.dt)), 40)
    srv = serving.Server(chunk_steps=7)
    stats = srv.run(jobs)
    assert stats["max_concurrent_jobs"] > 1          # their work overlapped
    bitwise = 0
    for j in jobs:
        ref = _alone(j)
        assert rel_l2(j.result, ref) <= 1e-12, j.jid
        bitwise += int(np.array_equal(j.result, ref))
    assert stats["p99_latency_s"] >= stats["p50_latency_s"] > 0
    print("bitwise equal:", bitwise, "of", len(jobs))


def test_admission_respects_budget():
    require_gpu()
    from paper_1903_04946_gb300 import serving
    jobs = serving.make_jobs(n_jobs=8, seed=5, load=8.0, max_points=1 << 12)
    for j in jobs:
        j.t = j.dt * min(int(round(j.t / j.dt)), 10)
    fps = [serving.footprint_bytes(j.problem, j.order, j.scheme) for j in jobs]
    # the biggest job fits only alone
    budget = max(fps) + min(fps) - 1
    srv = serving.Server(budget_bytes=budget, chunk_steps=5)
    stats = srv.run(jobs)
    assert stats["peak_footprint_bytes"] <= budget
    big = jobs[int(np.argmax(fps))]
    for j in jobs:
        if j is not big:
            assert j.finished <= big.admitted or big.finished <= j.admitted, j.jid
    assert all(j.result is not None and np.all(np.isfinite(j.result)) for j in jobs)


def test_cancellation_and_job_log(tmp_path):
    """A waiting job cancelled before admission is dropped; a running job
    cancelled mid-run is retired at its next chunk boundary without a result;
    every other job finishes as if alone; the log has one line per job."""
    require_gpu()
    import json

    from paper_1903_04946_gb300 import serving
    jobs = serving.make_jobs(n_jobs=6, seed=11, load=8.0, max_points=1 << 12)
    for j in jobs:
        j.t = j.dt * min(int(round(j.t / j.dt)), 40)
    srv = serving.Server(chunk_steps=2)
    srv.cancel(jobs[5].jid)
    target = jobs[0]

    def tick(server, now):
        if target.admitted >= 0 and target.steps_done > 0:
            server.cancel(target.jid)

    log = tmp_path / "jobs.jsonl"
    stats = srv.run(jobs, log=str(log), on_tick=tick)
    assert stats["cancelled"] == 2
    recs = {r["jid"]: r for r in map(json.loads, log.read_text().splitlines())}
    assert sorted(recs) == sorted(j.jid for j in jobs)
    assert recs[jobs[5].jid]["cancelled"] and recs[jobs[5].jid]["admitted_s"] < 0
    assert recs[target.jid]["cancelled"] and target.result is None
    assert recs[target.jid]["steps_done"] < target.steps_total
    for j in jobs[1:5]:
        r = recs[j.jid]
        assert not r["cancelled"] and abs(r["norm"] - 1.0) < 1e-10 and r["latency_s"] > 0
        assert rel_l2(j.result, _alone(j)) <= 1e-12
