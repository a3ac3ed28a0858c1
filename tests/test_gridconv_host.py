"""Host side of the grid-convergence study (App. B): the trigonometric
interpolation that compares wavefunctions on grids of different range and
density.  Checked against what fixes it: a band-limited periodic function is
reproduced exactly anywhere in its period, the samples themselves come back,
points outside the coarse range get zero, and a resolved Gaussian converges
exponentially with the number of samples."""
import numpy as np
import pytest

from paper_1903_04946_gb300.gridconv import grid_range, trig_interpolate


def test_band_limited_function_is_exact_between_samples():
    a, b, N = 3.0, 16.5, 64
    rng = np.random.default_rng(0)
    ks = np.arange(-N // 2 + 1, N // 2)                # strictly below Nyquist
    amp = rng.standard_normal(ks.size) + 1j * rng.standard_normal(ks.size)

    def f(x):
        return np.exp(2j * np.pi * np.outer(x - a, ks) / (b - a)) @ amp

    xs = a + (b - a) / N * np.arange(N)
    x = rng.uniform(a, b, size=200)
    got = trig_interpolate(f(xs), a, b, x)
    assert np.max(np.abs(got - f(x))) <= 1e-11 * np.max(np.abs(amp)) * ks.size


def test_samples_come_back_and_outside_is_zero():
    rng = np.random.default_rng(1)
    a, b, N = 0.5, 2.5, 32
    f = rng.standard_normal((2, N)) + 1j * rng.standard_normal((2, N))
    xs = a + (b - a) / N * np.arange(N)
    assert np.allclose(trig_interpolate(f, a, b, xs), f, rtol=0, atol=1e-13)
    out = trig_interpolate(f, a, b, np.array([a - 1e-9, b, b + 3.0]))
    assert np.all(out == 0)


def test_resolved_gaussian_converges_exponentially():
    x = np.linspace(-4.0, 4.0, 301)
    g = lambda q: np.exp(-q ** 2 / (2 * 0.6 ** 2))          # noqa: E731
    errs = []
    for N in (16, 24, 32, 48, 64):
        xs = -8.0 + 16.0 / N * np.arange(N)
        errs.append(np.max(np.abs(trig_interpolate(g(xs), -8.0, 8.0, x) - g(x))))
    assert errs[-1] < 1e-12
    assert all(e2 < e1 / 5 for e1, e2 in zip(errs[:-2], errs[1:-1]))


def test_grid_ranges_grow_by_sqrt2():
    assert grid_range(1024) == (3.0, 30.0)
    for N in (256, 512, 2048):
        a, b = grid_range(N)
        a2, b2 = grid_range(2 * N)
        assert a == a2 == 3.0
        assert (b2 - a2) / (b - a) == pytest.approx(np.sqrt(2.0), rel=1e-14)
