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
        assert j.problem.S * j.problem.n[0] <= 8192 and all(8 <= x <= 4096 for x in j.problem.n)


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
