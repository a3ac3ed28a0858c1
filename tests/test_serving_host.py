"""Host-side pieces of the serving loop (no GPU): the seeded job stream and
the device-memory footprint used for admission."""
import numpy as np

import synth


def test_job_stream_reproducible_and_mixed():
    from paper_1903_04946_gb300 import serving
    a = serving.make_jobs(n_jobs=20, seed=3)
    b = serving.make_jobs(n_jobs=20, seed=3)
    assert [j.problem.n for j in a] == [j.problem.n for j in b]
    assert [j.arrival for j in a] == [j.arrival for j in b]
    assert all(x.arrival < y.arrival for x, y in zip(a, a[1:]))
    assert len({j.problem.D for j in a}) > 1 and len({j.problem.S for j in a}) > 1
    for j in a:
        assert abs(j.t / j.dt - round(j.t / j.dt)) < 1e-12
        assert 500 - j.dt <= j.t <= 5000 + j.dt
        assert all(x >= 8 for x in j.problem.n) and 2 ** 8 <= j.problem.points <= 2 ** 21


def test_job_stream_spans_the_serving_configuration():
    # D in {1, 2, 3}, 2^8..2^21 points per surface, S in {2, 3, 4}: the draw
    # is not narrowed to any implementation limit (long axes included)
    jobs = [synth.serving_job(1907 + i)[0] for i in range(200)]
    assert {p.D for p in jobs} == {1, 2, 3}
    assert {p.S for p in jobs} == {2, 3, 4}
    logs = {int(np.log2(p.points)) for p in jobs}
    assert min(logs) == 8 and max(logs) == 21
    assert any(p.D == 1 and p.points > 8192 for p in jobs)
    assert any(max(p.n) > 4096 for p in jobs if p.D >= 2)
    assert any(p.S * p.n[0] > 8192 for p in jobs)


def test_footprint_grows_with_grid_order_and_surfaces():
    from paper_1903_04946_gb300 import serving
    small = synth.random_coupled(1, (32, 32), 2)
    big = synth.random_coupled(1, (64, 64), 2)
    three = synth.random_coupled(1, (32, 32), 3)
    f = serving.footprint_bytes
    assert f(big, 4) > f(small, 4)
    assert f(small, 8) > f(small, 4)
    assert f(three, 4) > f(small, 4)
    P = 32 * 32
    assert f(small, 2) >= 2 * 2 * P * 16 + 3 * P * 8


class _FakeContext:
    """Stands in for a library context: records the steps it is asked to
    propagate and reports itself busy for a few polls after each call."""
    live = 0

    def __init__(self, device=0, precision=0):
        _FakeContext.live += 1
        self.ctx = self
        self.steps = 0
        self.busy_polls = 0

    def load_problem(self, pr):
        self.pr = pr

    def propagate(self, t, dt):
        self.steps += int(round(t / dt))
        self.busy_polls = 2

    def psi(self):
        return np.zeros((self.pr.S,) + tuple(self.pr.n), dtype=np.complex128)

    def observables(self):
        return 1.0, 0.5, np.array([1.0] + [0.0] * (self.pr.S - 1))

    def close(self):
        _FakeContext.live -= 1


def _fake_busy(ctx):
    if ctx.busy_polls > 0:
        ctx.busy_polls -= 1
        return True
    return False


def test_scheduler_admission_cancellation_and_log(monkeypatch, tmp_path):
    """The serving loop's scheduling on the host: the admitted footprint never
    exceeds the budget, every job gets exactly its steps in chunks, a
    cancelled waiting job is never admitted, a job cancelled while running
    stops early without a result, and the log has one line per job."""
    import json

    from paper_1903_04946_gb300 import serving
    monkeypatch.setattr(serving, "Context", _FakeContext)
    monkeypatch.setattr(serving, "dso_busy", _fake_busy)
    monkeypatch.setattr(serving, "dso_set_scheme", lambda *a, **k: None)
    jobs = serving.make_jobs(n_jobs=12, seed=21, load=50.0, max_points=1 << 12)
    for j in jobs:
        j.t = j.dt * min(int(round(j.t / j.dt)), 30)
    fps = [serving.footprint_bytes(j.problem, j.order, j.scheme) for j in jobs]
    budget = 3 * max(fps)
    srv = serving.Server(budget_bytes=budget, chunk_steps=4, slots=False)
    srv.cancel(jobs[11].jid)
    running = jobs[2]

    def tick(server, now):
        if running.steps_done >= 4:
            server.cancel(running.jid)

    log = tmp_path / "log.jsonl"
    stats = srv.run(jobs, log=str(log), on_tick=tick)
    assert stats["peak_footprint_bytes"] <= budget
    assert stats["cancelled"] == 2 and _FakeContext.live == 0
    recs = {r["jid"]: r for r in map(json.loads, log.read_text().splitlines())}
    assert sorted(recs) == sorted(j.jid for j in jobs)
    assert recs[jobs[11].jid]["admitted_s"] < 0 and recs[jobs[11].jid]["cancelled"]
    assert recs[running.jid]["cancelled"] and running.result is None
    assert 4 <= running.steps_done < running.steps_total
    for j in jobs:
        if j.cancelled:
            continue
        assert j.steps_done == j.steps_total and j.result is not None
        assert recs[j.jid]["norm"] == 1.0 and recs[j.jid]["latency_s"] >= 0


class _FakeBatch:
    """Stands in for a batch: every step advances each unfinished slot by one
    composed step and reports itself busy for a poll; jobs above 2^10 points
    are refused (too large for a slot), so they take the per-job path."""

    def __init__(self, device=0, precision=0):
        self.slots, self.next, self.busy_polls, self.launches = {}, 0, 0, 0

    def add(self, ctx, t, dt):
        from paper_1903_04946_gb300 import DSOError
        if ctx.pr.points > 1 << 10:
            raise DSOError(-1, "dso_batch_add")
        slot = self.next
        self.next += 1
        self.slots[slot] = [0, int(round(t / dt))]
        return slot

    def step(self):
        for s in self.slots.values():
            if s[0] < s[1]:
                s[0] += 1
        self.busy_polls = 1
        self.launches += 1
        return sum(1 for s in self.slots.values() if s[0] < s[1])

    def busy(self):
        if self.busy_polls > 0:
            self.busy_polls -= 1
            return True
        return False

    def status(self, slot):
        return tuple(self.slots[slot])

    def retire(self, slot):
        del self.slots[slot]


def test_scheduler_with_batch_slots(monkeypatch):
    """Jobs that fit a slot advance one step per batch round; the others
    fall back to their own chunked propagation; every job gets exactly its
    steps, a job cancelled while in a slot leaves at a step boundary."""
    from paper_1903_04946_gb300 import serving
    monkeypatch.setattr(serving, "Context", _FakeContext)
    monkeypatch.setattr(serving, "Batch", _FakeBatch)
    monkeypatch.setattr(serving, "dso_busy", _fake_busy)
    monkeypatch.setattr(serving, "dso_set_scheme", lambda *a, **k: None)
    jobs = serving.make_jobs(n_jobs=16, seed=23, load=50.0, max_points=1 << 12)
    for j in jobs:
        j.t = j.dt * min(int(round(j.t / j.dt)), 12)
    srv = serving.Server(budget_bytes=1 << 40, chunk_steps=5)
    small = [j for j in jobs if j.problem.points <= 1 << 10]
    big = [j for j in jobs if j.problem.points > 1 << 10]
    assert small and big
    victim = small[0]

    def tick(server, now):
        if victim.slot >= 0 and victim.steps_done >= 2:
            server.cancel(victim.jid)

    stats = srv.run(jobs, on_tick=tick)
    assert _FakeContext.live == 0
    assert victim.cancelled and victim.result is None and 2 <= victim.steps_done < victim.steps_total
    for j in jobs:
        if j is victim:
            continue
        assert j.steps_done == j.steps_total and j.result is not None, j.jid
    # slotted jobs never took the per-job path
    assert stats["batch_launches"] >= max(j.steps_total for j in small if j is not victim)
