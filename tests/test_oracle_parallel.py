"""The OpenMP build of the oracle (the benchmark's parallel CPU line) gives
the same bits as the single-threaded build.

It splits only loops whose iterations are independent: the vertices of one
colour in a sweep (never neighbours), the rows of y = A x, and the fine rows
of the prolongation.  No sum changes order, so solution, iteration count and
every single step must be bitwise equal.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2505_09064_gb300 import meshgen

CASES = {
    "2d_n48": dict(dim=2, n=48, jitter=0.2, seed=31, checker=True, E=100.0),
    "3d_n10": dict(dim=3, n=10, jitter=0.15, seed=32, nu=0.4),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_parallel_oracle_bitwise_equal(name):
    p = meshgen.make_problem(None, **CASES[name])
    o1 = oracle.Oracle(p)
    o4 = oracle.Oracle(p, threads=4)
    assert o1.threads == 1 and o4.threads == 4
    F = o1.assemble_load(p["body_force"])
    F[p["dirichlet_dofs"]] = 0.0
    U1, it1, rr1, st1, _ = o1.solve(F, tol=1e-8)
    U4, it4, rr4, st4, _ = o4.solve(F, tol=1e-8)
    assert st1 == st4 == 0 and it1 == it4 and rr1 == rr4
    assert np.array_equal(U1, U4)
    rs = meshgen.Stream(7)
    for l in range(o1.num_levels - 1):
        nl = o1.level_info(l)[0] * p["dim"]
        x = rs.uniform(nl, -1.0, 1.0)
        assert np.array_equal(o1.apply_A(l, x), o4.apply_A(l, x))
        b = rs.uniform(nl, -1.0, 1.0)
        x0 = rs.uniform(nl, -1.0, 1.0)
        for fwd in (True, False):
            assert np.array_equal(o1.gs_sweep(l, b, x0, forward=fwd), o4.gs_sweep(l, b, x0, forward=fwd))
        nc = o1.level_info(l + 1)[0] * p["dim"]
        ec = rs.uniform(nc, -1.0, 1.0)
        assert np.array_equal(o1.prolong_add(l, ec, b), o4.prolong_add(l, ec, b))


@pytest.mark.parametrize("name", sorted(CASES))
def test_parallel_oracle_cycle_variants_bitwise_equal(name):
    """The W-cycle, the additive form and the lexicographic smoother go
    through the same parallel loops; both builds still agree bit for bit."""
    p = meshgen.make_problem(None, **CASES[name])
    o1 = oracle.Oracle(p)
    o4 = oracle.Oracle(p, threads=4)
    F = o1.assemble_load(p["body_force"])
    F[p["dirichlet_dofs"]] = 0.0
    for kw, smoother in [(dict(gamma=2), "multicolour"), (dict(additive=True), "multicolour"),
                         (dict(gamma=1), "lexicographic")]:
        for o in (o1, o4):
            o.set_cycle(**kw)
            o.set_smoother(smoother)
        U1, it1, rr1, st1, _ = o1.solve(F, tol=1e-8)
        U4, it4, rr4, st4, _ = o4.solve(F, tol=1e-8)
        assert st1 == st4 == 0 and it1 == it4 and rr1 == rr4
        assert np.array_equal(U1, U4), (kw, smoother)
