"""Robustness of the iteration count: mesh size and Poisson ratio.

Thm. 4.1 bounds the condition number of the preconditioned system
independently of the mesh size, so PCG iterations to a fixed relative
residual should stay nearly flat as the mesh is refined; Sec. 5 reports the
same for several Poisson ratios.  Each case below solves the jittered unit
square (2D) or cube (3D) recipe, clamped on x = 0, with the body-force load,
through the library, and checks that the iteration count grows by at most a
small factor from the coarsest to the finest mesh of a series.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2505_09064_gb300 import meshgen, vasmg  # noqa: E402

pytestmark = pytest.mark.gpu

SERIES = {
    # (dim, grid sides)
    "2d": (2, [33, 65, 129, 257, 513]),
    "3d": (3, [9, 17, 33, 49]),
}
NUS = [0.1, 0.3, 0.45]


@pytest.fixture(scope="module")
def built():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)
    return True


def _iterations(dim, n, nu, precision):
    prob = meshgen.make_problem(None, dim=dim, n=n, jitter=0.2 if dim == 2 else 0.15, seed=40 + n, E=1.0, nu=nu)
    s = vasmg.Solver(prob, precision=precision, stream=torch.cuda.current_stream().cuda_stream)
    try:
        ndof = prob["coords"].shape[0] * dim
        F = torch.zeros(ndof, dtype=torch.float64, device="cuda")
        s.assemble_load(prob["body_force"], F)
        U = torch.zeros_like(F)
        rc, st, _ = s.solve(F, U, 1e-6)
        assert rc == 0 and st.rel_res < 1e-6
        return st.iterations
    finally:
        s.close()


@pytest.mark.parametrize("series", sorted(SERIES))
@pytest.mark.parametrize("nu", NUS)
def test_iterations_nearly_flat_under_refinement(built, series, nu):
    dim, sides = SERIES[series]
    its = [_iterations(dim, n, nu, "fp32") for n in sides]
    print(f"\n{series} nu={nu}: " + ", ".join(f"n={n}: {k}" for n, k in zip(sides, its)))
    # at most 2x from the coarsest to the finest mesh, and no blow-up
    assert max(its) <= 2 * min(its) + 4, its
    assert its[-1] <= 2 * its[0] + 4, its
