"""Host logic of the time-to-1e-10 study, with the GPU propagation replaced
by a model: job j's error at dt = t_f / 2^k is c_j 2^(-order k) 1e4 and a
run costs a fixed time per substep, 0.4x per job when batched.  The study
must find each job's smallest k, group the jobs by it, and report the
shared-dt and grouped batches and the single path consistently."""
import numpy as np
import pytest

from paper_1903_04946_gb300 import efficiency as E


def _setup(monkeypatch, batch):
    coef = {}

    def err_model(j, order, k):
        return (1.0 + 3.0 * j / batch) * 2.0 ** (-order * k) * 1e4

    def fake_propagate(problems, scheme, order, tf, k, batched):
        ids = [coef.setdefault(id(p), len(coef)) for p in problems]
        nsub = len(E.dso_scheme_coefficients(order, E._code(scheme))[1])
        secs = 1e-6 * nsub * 2 ** k * (0.4 * len(problems) if batched else 1.0)
        if scheme == "suzuki" and order == 10 and k == 8:   # the reference run (ref_k + 1): exact
            return np.zeros(len(problems)), secs
        return np.array([err_model(j, order, k) for j in ids]), secs

    monkeypatch.setattr(E, "_propagate", fake_propagate)
    monkeypatch.setattr(E, "_err", lambda problem, psi, ref: float(np.ravel(psi)[0] - np.ravel(ref)[0]))
    return err_model


def test_study_groups_jobs_by_the_dt_they_need(monkeypatch):
    batch = 8
    err_model = _setup(monkeypatch, batch)
    out = E.study(grid=8, batch=batch, kmax=20, ref_k=7)
    rows = {(r["scheme"], r["order"]): r for r in out["methods"]}
    assert rows[("triple_jump", 2)]["reached"] is False       # needs k > 20
    for (scheme, order), r in rows.items():
        if not r.get("batch_reached"):
            continue
        need = [min(k for k in range(2, 40) if err_model(j, order, k) <= 1e-10) for j in range(batch)]
        groups = {}
        for k in need:
            groups[str(k)] = groups.get(str(k), 0) + 1
        assert r["grouped_sizes_by_k"] == groups, (scheme, order)
        assert r["batch_k"] == max(need)
        # the grouped batch costs what its groups cost; the shared one runs all at the largest k
        nsub = r["substeps_per_step"]
        grouped = sum(1e-6 * nsub * 2 ** int(k) * 0.4 * cnt for k, cnt in groups.items()) / batch
        assert r["grouped_batch_per_wavepacket_seconds"] == pytest.approx(grouped, rel=1e-12)
        assert r["batch_per_wavepacket_seconds"] == pytest.approx(1e-6 * nsub * 2 ** max(need) * 0.4, rel=1e-12)
        single_avg = np.mean([1e-6 * nsub * 2 ** k for k in need])
        assert r["single_avg_seconds"] == pytest.approx(single_avg, rel=1e-12)
    assert out["grouped_batch_vs_single_speedup"] == pytest.approx(1 / 0.4, rel=1e-9)
