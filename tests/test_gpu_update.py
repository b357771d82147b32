"""Reusing a hierarchy for new material data or new Dirichlet values.

The tree, transfers, patterns, colourings and the solve engine's layout
depend only on the mesh and on which dofs are constrained, so
vasmg_update_data recomputes values only.  A handle set up with one material
and updated to another must then solve exactly like a handle set up with the
second material from scratch: same iteration count, same solution (bitwise:
the same kernels run on the same values in the same order).  The updated
handle's FP64 solve is also compared with the CPU oracle set up from scratch
on the new data (assembly of Sec. 2, Galerkin products eq. (Ac)): iterations
+-1, solution to 1e-10 (max norm).
"""
from __future__ import annotations

import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2505_09064_gb300 import meshgen, vasmg  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def built():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)
    return True


def _variant(p, seed, nonhomogeneous):
    """Same mesh and constrained dofs; per-element E in [1, 100], new nu, and
    optionally non-zero Dirichlet values."""
    q = dict(p)
    ne = p["elems"].shape[0]
    rs = meshgen.Stream(seed)
    E = 1.0 + 99.0 * rs.uniform(ne)
    nu = 0.2 + 0.25 * rs.uniform(1)[0]
    q["lam"], q["mu"] = meshgen.lame(E, np.full(ne, nu))
    if nonhomogeneous:
        q["dirichlet_values"] = rs.uniform(p["dirichlet_dofs"].size, -0.01, 0.01)
    return q


def _solve(s, F):
    Fd = torch.tensor(F, dtype=torch.float64, device="cuda")
    Ud = torch.zeros_like(Fd)
    rc, st, _ = s.solve(Fd, Ud, 1e-8)
    assert rc == 0
    return Ud.cpu().numpy(), st.iterations


@pytest.mark.parametrize("dim,n", [(2, 60), (3, 12)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("nonhomogeneous", [False, True])
def test_update_equals_fresh_setup(built, dim, n, precision, nonhomogeneous):
    p = meshgen.make_problem(None, dim=dim, n=n, jitter=0.2 if dim == 2 else 0.15, seed=70 + n)
    q = _variant(p, 71 + n, nonhomogeneous)
    stream = torch.cuda.current_stream().cuda_stream
    ndof = p["coords"].shape[0] * dim
    F = meshgen.Stream(72).uniform(ndof, -1.0, 1.0)
    s = vasmg.Solver(p, precision=precision, stream=stream)
    fresh = vasmg.Solver(q, precision=precision, stream=stream)
    try:
        _solve(s, F)  # solve once with the old data (graphs built, buffers warm)
        t0 = time.perf_counter()
        s.update(q)
        t_update = time.perf_counter() - t0
        U1, it1 = _solve(s, F)
        U2, it2 = _solve(fresh, F)
        assert it1 == it2
        assert np.array_equal(U1, U2)
        # and the update really changed the operator
        U0, _ = _solve(vasmg.Solver(p, precision=precision, stream=stream), F)
        assert not np.allclose(U0, U1)
        print(f"\nupdate {1e3 * t_update:.1f} ms")
    finally:
        s.close()
        fresh.close()


@pytest.mark.parametrize("dim,n", [(2, 60), (3, 12)])
@pytest.mark.parametrize("nonhomogeneous", [False, True])
def test_update_matches_oracle_on_new_data(built, dim, n, nonhomogeneous):
    p = meshgen.make_problem(None, dim=dim, n=n, jitter=0.2 if dim == 2 else 0.15, seed=80 + n)
    q = _variant(p, 81 + n, nonhomogeneous)
    stream = torch.cuda.current_stream().cuda_stream
    ndof = p["coords"].shape[0] * dim
    F = meshgen.Stream(82).uniform(ndof, -1.0, 1.0)
    s = vasmg.Solver(p, precision="fp64", stream=stream)
    try:
        _solve(s, F)
        s.update(q)
        U1, it1 = _solve(s, F)
        o = oracle.Oracle(q)
        U_ref, it_ref, _, st_ref, _ = o.solve(F, tol=1e-8)
        assert st_ref == 0
        assert abs(it1 - it_ref) <= 1, (it1, it_ref)
        err = float(np.max(np.abs(U1 - U_ref)) / np.max(np.abs(U_ref)))
        assert err <= 1e-10, err
        if nonhomogeneous:
            # the new Dirichlet values are written into U
            assert np.array_equal(U1[q["dirichlet_dofs"]], q["dirichlet_values"])
    finally:
        s.close()
