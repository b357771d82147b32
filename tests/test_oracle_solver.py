"""Pins for the oracle's smoother, V-cycle, coarsest solve and PCG (Alg. 1-3)
against dense linear algebra (numpy), scipy's CG, the colouring's defining
properties and the near-constant iteration count that Theorem 4.1 predicts."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from paper_2505_09064_gb300 import meshgen
from tests.helpers import dense_from_bsr


def _prob(dim, n, seed, **kw):
    return meshgen.make_problem(None, dim=dim, n=n, seed=seed, jitter=0.2 if dim == 2 else 0.15, **kw)


def _reduced_rhs(o, p):
    F = o.assemble_load(p["body_force"])
    F[p["dirichlet_dofs"]] = 0.0
    return F


def _priority(o, l, nv, dim):
    """Colouring priority: splitmix64 on the fine level; on coarser levels the
    lattice class sum_a ((p_a/u) mod 3) 3^a first (class 0 highest), u the
    side of the level's smallest cell."""
    from tests.helpers import K_of, deinterleave

    sm = meshgen.splitmix64(np.arange(nv, dtype=np.uint64))
    if l == 0:
        return sm
    K = K_of(dim)
    D = int(o.cells(l)[:, 0].max())
    q = deinterleave(o.lattice(l), dim, K + 1) >> np.uint64(K - D)
    cls = np.zeros(nv, dtype=np.uint64)
    w = 1
    for a in range(dim):
        cls += (q[:, a] % np.uint64(3)) * np.uint64(w)
        w *= 3
    return ((np.uint64(w - 1) - cls) << np.uint64(58)) | (sm >> np.uint64(6))


@pytest.mark.parametrize("dim,n,seed", [(2, 10, 1), (3, 5, 2)])
def test_colouring_is_proper_and_greedy_by_priority(oracle_mod, dim, n, seed):
    p = _prob(dim, n, seed)
    o = oracle_mod.Oracle(p)
    for l in range(o.num_levels):
        rp, ci, _ = o.operator(l)
        col = o.colours(l)
        nv = len(rp) - 1
        prio = _priority(o, l, nv, dim)
        for i in range(nv):
            nb = ci[rp[i]:rp[i + 1]]
            nb = nb[nb != i]
            assert not np.any(col[nb] == col[i])
            higher = nb[(prio[nb] > prio[i]) | ((prio[nb] == prio[i]) & (nb < i))]
            used = set(col[higher].tolist())
            smallest = next(c for c in range(len(used) + 1) if c not in used)
            assert col[i] == smallest


def test_coarse_levels_use_3_to_the_d_colours(oracle_mod):
    """Jittered meshes give radius-2 Galerkin stencils on the uniform coarse
    levels; the class-first priority then colours them with exactly 3^d colours
    (a 3^d block of lattice points is a clique, so this is optimal)."""
    for dim, n in [(2, 65), (3, 17)]:
        p = _prob(dim, n, 1)
        o = oracle_mod.Oracle(p)
        checked = 0
        for l in range(2, o.num_levels):
            nv, _, ncol = o.level_info(l)
            if nv >= 7 ** dim:
                assert ncol == 3 ** dim, (dim, l, ncol)
                checked += 1
        assert checked >= 1


@pytest.mark.parametrize("dim,n,seed", [(2, 8, 3), (3, 4, 4)])
def test_gs_sweep_equals_dense_triangular_solve(oracle_mod, dim, n, seed):
    """One forward sweep from x0: (D + L_c) x1 = b - U_c x0 with L_c / U_c the
    block-lower / upper parts in colour order; a backward sweep swaps them."""
    p = _prob(dim, n, seed)
    o = oracle_mod.Oracle(p)
    rs = meshgen.Stream(17)
    for l in range(min(2, o.num_levels)):
        rp, ci, v = o.operator(l)
        A = dense_from_bsr(rp, ci, v, dim)
        col = o.colours(l)
        nv = len(rp) - 1
        ncol = col.max() + 1
        # colour rank of every dof
        rank = np.repeat(col, dim)
        same_vertex = np.repeat(np.arange(nv), dim)
        Dm = np.where(same_vertex[:, None] == same_vertex[None, :], A, 0.0)
        lower = (rank[:, None] > rank[None, :])
        upper = (rank[:, None] < rank[None, :])
        b = rs.uniform(nv * dim, -1, 1)
        x0 = rs.uniform(nv * dim, -1, 1)
        xf = o.gs_sweep(l, b, x0, forward=True)
        ref_f = np.linalg.solve(Dm + A * lower, b - (A * upper) @ x0)
        np.testing.assert_allclose(xf, ref_f, rtol=1e-10, atol=1e-10 * np.abs(ref_f).max())
        xb = o.gs_sweep(l, b, x0, forward=False)
        ref_b = np.linalg.solve(Dm + A * upper, b - (A * lower) @ x0)
        np.testing.assert_allclose(xb, ref_b, rtol=1e-10, atol=1e-10 * np.abs(ref_b).max())
        assert ncol >= 2


@pytest.mark.parametrize("dim,n,seed", [(2, 9, 5), (3, 5, 6)])
def test_vcycle_is_symmetric_positive_definite(oracle_mod, dim, n, seed):
    p = _prob(dim, n, seed)
    o = oracle_mod.Oracle(p)
    nv = p["coords"].shape[0]
    rs = meshgen.Stream(23)
    dirm = np.zeros(nv * dim, bool)
    dirm[p["dirichlet_dofs"]] = True
    for _ in range(4):
        x = rs.uniform(nv * dim, -1, 1)
        y = rs.uniform(nv * dim, -1, 1)
        x[dirm] = 0
        y[dirm] = 0
        Mx, My = o.vcycle(x), o.vcycle(y)
        assert abs(x @ My - y @ Mx) <= 1e-12 * np.sqrt((x @ Mx) * (y @ My))
        assert x @ Mx > 0


def test_coarsest_solve_equals_dense_direct(oracle_mod):
    for dim, n in [(2, 9), (3, 5)]:
        p = _prob(dim, n, 3)
        o = oracle_mod.Oracle(p)
        L = o.num_levels - 1
        rp, ci, v = o.operator(L)
        A = dense_from_bsr(rp, ci, v, dim)
        b = meshgen.Stream(5).uniform(A.shape[0], -1, 1)
        np.testing.assert_allclose(o.coarse_solve(b), np.linalg.solve(A, b), rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("dim,n,seed", [(2, 12, 7), (2, 16, 8), (3, 6, 9)])
def test_pcg_solution_equals_dense_direct_solve(oracle_mod, dim, n, seed):
    p = _prob(dim, n, seed, E=7.0, nu=0.33)
    o = oracle_mod.Oracle(p)
    rp, ci, v = o.operator(0)
    A = dense_from_bsr(rp, ci, v, dim)
    F = _reduced_rhs(o, p)
    Uref = np.linalg.solve(A, F)
    U, it, rr, st, hist = o.solve(F, tol=1e-12, hist_cap=200)
    assert st == 0 and rr < 1e-12
    kappa = np.linalg.cond(A)
    err = np.linalg.norm(U - Uref) / np.linalg.norm(Uref)
    assert err <= 1e-12 * kappa
    # the recorded history is the relative residual of the recursive residual
    assert np.all(np.diff(np.log(hist)) < 0.5)


def test_unpreconditioned_pcg_is_textbook_cg(oracle_mod):
    p = _prob(2, 12, 4)
    o = oracle_mod.Oracle(p)
    rp, ci, v = o.operator(0)
    A = dense_from_bsr(rp, ci, v, 2)
    F = _reduced_rhs(o, p)
    U, it, rr, st, _ = o.solve(F, tol=1e-8, precondition=False, max_iters=5000)
    count = [0]

    def cb(_):
        count[0] += 1

    Us, info = spla.cg(sp.csr_matrix(A), F, rtol=1e-8, atol=0.0, maxiter=5000, callback=cb)
    assert st == 0 and info == 0
    assert abs(it - count[0]) <= 1
    np.testing.assert_allclose(U, Us, rtol=0, atol=1e-7 * np.abs(Us).max())


def test_zero_rhs_returns_zero_iterations(oracle_mod):
    p = _prob(2, 6, 1)
    o = oracle_mod.Oracle(p)
    U, it, rr, st, _ = o.solve(np.zeros(p["coords"].shape[0] * 2))
    assert it == 0 and st == 0 and np.all(U == 0)


@pytest.mark.slow
def test_iterations_nearly_flat_under_refinement(oracle_mod):
    """Theorem 4.1: kappa(B_h A_h) = O(1), so the iteration count barely moves
    as the mesh is refined (the paper reports 9-12 iterations for its 2D
    examples)."""
    its = []
    for n in (17, 33, 65, 129):
        p = _prob(2, n, 1)
        o = oracle_mod.Oracle(p)
        F = _reduced_rhs(o, p)
        _, it, rr, st, _ = o.solve(F, tol=1e-6)
        assert st == 0
        its.append(it)
    assert max(its) <= 16 and max(its) - min(its) <= 5, its


@pytest.mark.parametrize("dim,n,seed", [(2, 8, 31), (3, 4, 32)])
def test_lexicographic_sweep_equals_dense_triangular_solve(oracle_mod, dim, n, seed):
    """The paper's smoother (Sec. 2.1, Alg. 1): scalar Gauss-Seidel with the
    unknowns in component-major order.  Writing A in that order as
    L + D + U (scalar strictly lower, diagonal, strictly upper), one forward
    sweep from x0 solves (D + L) x1 = b - U x0; a backward sweep swaps L, U."""
    p = _prob(dim, n, seed)
    o = oracle_mod.Oracle(p)
    o.set_smoother("lexicographic")
    rs = meshgen.Stream(41)
    for l in range(min(2, o.num_levels)):
        rp, ci, v = o.operator(l)
        A = dense_from_bsr(rp, ci, v, dim)  # vertex-major dofs: vertex * dim + a
        nv = len(rp) - 1
        # position of vertex-major dof (i, a) in component-major order
        pos = np.array([a * nv + i for i in range(nv) for a in range(dim)])
        lower = pos[:, None] > pos[None, :]
        upper = pos[:, None] < pos[None, :]
        Dg = np.diag(np.diag(A))
        b = rs.uniform(nv * dim, -1, 1)
        x0 = rs.uniform(nv * dim, -1, 1)
        xf = o.gs_sweep(l, b, x0, forward=True)
        ref_f = np.linalg.solve(Dg + A * lower, b - (A * upper) @ x0)
        np.testing.assert_allclose(xf, ref_f, rtol=1e-10, atol=1e-10 * np.abs(ref_f).max())
        xb = o.gs_sweep(l, b, x0, forward=False)
        ref_b = np.linalg.solve(Dg + A * upper, b - (A * lower) @ x0)
        np.testing.assert_allclose(xb, ref_b, rtol=1e-10, atol=1e-10 * np.abs(ref_b).max())


@pytest.mark.parametrize("dim,n,seed", [(2, 9, 5), (3, 5, 6)])
def test_lexicographic_vcycle_symmetric_and_solves(oracle_mod, dim, n, seed):
    """With forward pre- and backward post-smoothing the lexicographic V-cycle
    is symmetric positive definite too, and PCG with it reaches the dense
    direct solution."""
    p = _prob(dim, n, seed)
    o = oracle_mod.Oracle(p)
    o.set_smoother("lexicographic")
    nv = p["coords"].shape[0]
    rs = meshgen.Stream(43)
    dirm = np.zeros(nv * dim, bool)
    dirm[p["dirichlet_dofs"]] = True
    for _ in range(3):
        x = rs.uniform(nv * dim, -1, 1)
        y = rs.uniform(nv * dim, -1, 1)
        x[dirm] = 0
        y[dirm] = 0
        Mx, My = o.vcycle(x), o.vcycle(y)
        assert abs(x @ My - y @ Mx) <= 1e-12 * np.sqrt((x @ Mx) * (y @ My))
        assert x @ Mx > 0
    F = o.assemble_load(p["body_force"])
    U, it, rr, st, _ = o.solve(F, tol=1e-10)
    assert st == 0 and it > 0
    rp, ci, v = o.operator(0)
    A = dense_from_bsr(rp, ci, v, dim)
    Fr = F.copy()
    Fr[dirm] = 0.0
    Uref = np.linalg.solve(A, Fr)
    assert np.abs(U - Uref).max() <= 1e-8 * np.abs(Uref).max()


@pytest.mark.parametrize("dim,n,seed", [(2, 33, 61), (3, 9, 62)])
def test_multicolour_costs_few_iterations_over_lexicographic(oracle_mod, dim, n, seed):
    """The GPU path's smoother (multicolour point-block GS) against the
    paper's (scalar lexicographic GS, Sec. 2.1): on the same hierarchy both
    V-cycle preconditioners converge, within a few iterations of each other."""
    p = _prob(dim, n, seed)
    o = oracle_mod.Oracle(p)
    F = o.assemble_load(p["body_force"])
    its = {}
    for sm in ("multicolour", "lexicographic"):
        o.set_smoother(sm)
        _, it, rr, st, _ = o.solve(F, tol=1e-6)
        assert st == 0 and rr < 1e-6
        its[sm] = it
    assert abs(its["multicolour"] - its["lexicographic"]) <= 4, its
