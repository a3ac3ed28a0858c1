"""The grid-convergence study (App. B) on the GPU: the error of the
wavefunction propagated on coarser grids, measured on the finest grid by
trigonometric interpolation, falls by orders of magnitude per doubling of
the grid (exponential convergence); the initial packet is resolved on every
grid (its error is round-off); and the error of representing the converged
result on the coarse grid is of the same size as the total error."""
import pytest

from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def test_grid_convergence_is_exponential():
    require_gpu()
    from paper_1903_04946_gb300 import gridconv
    out = gridconv.study(tf=500.0, nmax=2048, nmin=256, k=6)
    rows = out["grids"]
    assert [r["N"] for r in rows] == [256, 512, 1024]
    e = [r["final"]["total_error"] for r in rows]
    assert e[0] > 1e3 * e[1] and e[1] > 1e3 * e[2], e    # oracle run of the same study: 1.4e-3, 1.3e-7, 1.1e-13
    assert all(r["initial"]["total_error"] < 1e-12 for r in rows)
    assert all(0.3 <= r["final"]["ratio"] <= 1.5 for r in rows)
