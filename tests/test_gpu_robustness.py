"""Robustness of the iteration count: mesh size and Poisson ratio.

Thm. 4.1 bounds the condition number of the preconditioned system
independently of the mesh size, so PCG iterations to a fixed relative
residual should stay nearly flat as the mesh is refined; Sec. 5 reports the
same for several Poisson ratios (nu = 0.1, 0.2, 0.3, 0.4, 0.45).  Each case
below solves the jittered unit square (2D) or cube (3D) recipe, clamped on
x = 0, with the body-force load, through the library:

  - FP32 V-cycle, the full series: the iteration count grows by at most a
    small factor from the coarsest to the finest mesh;
  - FP64, on the sizes the oracle reaches (2D 33^2-129^2, 3D 9^3-17^3): the
    iteration count equals the oracle's +-1 and the solution matches it to
    1e-10 (max norm), for every nu.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2505_09064_gb300 import meshgen, vasmg  # noqa: E402

pytestmark = pytest.mark.gpu

SERIES = {
    # (dim, grid sides)
    "2d": (2, [33, 65, 129, 257, 513]),
    "3d": (3, [9, 17, 33, 49]),
}
NUS = [0.1, 0.2, 0.3, 0.4, 0.45]
ORACLE_SIDES = {2: [33, 65, 129], 3: [9, 13, 17]}


@pytest.fixture(scope="module")
def built():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)
    return True


def _problem(dim, n, nu):
    return meshgen.make_problem(None, dim=dim, n=n, jitter=0.2 if dim == 2 else 0.15, seed=40 + n, E=1.0, nu=nu)


def _iterations(dim, n, nu, precision):
    prob = _problem(dim, n, nu)
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


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("nu", NUS)
def test_fp64_iterations_match_oracle_over_nu(built, dim, nu):
    """Thm. 4.1's mesh-independent bound is a property of the method, so the
    library must reproduce the oracle's counts, not only their trend."""
    rows = []
    for n in ORACLE_SIDES[dim]:
        prob = _problem(dim, n, nu)
        o = oracle.Oracle(prob)
        F = o.assemble_load(prob["body_force"])
        U_ref, it_ref, _, st_ref, _ = o.solve(F, tol=1e-6)
        assert st_ref == 0
        s = vasmg.Solver(prob, precision="fp64", stream=torch.cuda.current_stream().cuda_stream)
        try:
            Fd = torch.from_numpy(F).cuda()
            U = torch.zeros_like(Fd)
            rc, st, _ = s.solve(Fd, U, 1e-6)
            assert rc == 0
            err = float(np.max(np.abs(U.cpu().numpy() - U_ref)) / np.max(np.abs(U_ref)))
            assert abs(st.iterations - it_ref) <= 1, (n, st.iterations, it_ref)
            assert err <= 1e-10, (n, err)
            rows.append((n, st.iterations, it_ref))
        finally:
            s.close()
    print(f"\n{dim}D nu={nu}: " + ", ".join(f"n={n}: {a} (oracle {b})" for n, a, b in rows))
