"""Pins for the oracle's P1 elasticity assembly (Sec. 2) against facts that do
not come from the oracle itself: the textbook Voigt form B^T D B, the paper's
own 2x2 block form, the rigid-body null space, exact symmetry, the total load,
the load's distribution over the vertices (one-element closed form and the
first-moment identity), and the linear-displacement patch test."""
import numpy as np
import pytest

from paper_2505_09064_gb300 import meshgen
from tests.helpers import dense_from_bsr, rigid_modes, voigt_element_stiffness


def _single_element(dim, seed):
    rs = meshgen.Stream(seed)
    X = rs.uniform((dim + 1) * dim, -1, 1).reshape(dim + 1, dim)
    sign = np.linalg.det((X[1:] - X[0]).T)
    if sign < 0:
        X[[1, 2]] = X[[2, 1]]
    lam, mu = rs.uniform(2, 0.5, 3.0)
    elems = np.arange(dim + 1, dtype=np.int32)[None, :]
    return dict(dim=dim, coords=X, elems=elems, lam=np.array([lam]), mu=np.array([mu]),
                dirichlet_dofs=np.zeros(0, np.int64), dirichlet_values=None, body_force=np.zeros(dim))


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_single_element_matches_voigt_form(oracle_mod, dim, seed):
    p = _single_element(dim, seed)
    o = oracle_mod.Oracle(p, coarse_max_dofs=100)
    rp, ci, v = o.operator(0)
    A = dense_from_bsr(rp, ci, v, dim)
    Kref = voigt_element_stiffness(p["coords"], p["lam"][0], p["mu"][0])
    np.testing.assert_allclose(A, Kref, rtol=1e-13, atol=1e-13 * np.abs(Kref).max())


def test_block_form_of_the_paper_2d(oracle_mod):
    """A = [[(lam+2mu)A11 + mu A22, lam A12 + mu A21], [lam A21 + mu A12,
    (lam+2mu)A22 + mu A11]] in component-major order (Sec. 2)."""
    p = meshgen.make_problem(None, dim=2, n=6, jitter=0.2, seed=5, E=3.0, nu=0.3)
    p["dirichlet_dofs"] = np.zeros(0, np.int64)
    lam, mu = p["lam"][0], p["mu"][0]
    o = oracle_mod.Oracle(p, coarse_max_dofs=10000)
    rp, ci, v = o.operator(0)
    A = dense_from_bsr(rp, ci, v, 2)
    X, E = p["coords"], p["elems"]
    N = X.shape[0]
    A11, A12, A21, A22 = (np.zeros((N, N)) for _ in range(4))
    for e in E:
        J = (X[e[1:]] - X[e[0]]).T
        G = np.linalg.inv(J)
        g = np.vstack([-G.sum(0), G])
        area = abs(np.linalg.det(J)) / 2
        for r in range(3):
            for c in range(3):
                A11[e[r], e[c]] += area * g[r, 0] * g[c, 0]
                A12[e[r], e[c]] += area * g[r, 0] * g[c, 1]
                A21[e[r], e[c]] += area * g[r, 1] * g[c, 0]
                A22[e[r], e[c]] += area * g[r, 1] * g[c, 1]
    paper = np.block([[(lam + 2 * mu) * A11 + mu * A22, lam * A12 + mu * A21],
                      [lam * A21 + mu * A12, (lam + 2 * mu) * A22 + mu * A11]])
    perm = np.concatenate([np.arange(N) * 2, np.arange(N) * 2 + 1])  # component-major
    np.testing.assert_allclose(A[np.ix_(perm, perm)], paper, rtol=1e-12, atol=1e-12 * np.abs(paper).max())


@pytest.mark.parametrize("dim,n", [(2, 9), (3, 5)])
def test_rigid_body_null_space_and_symmetry(oracle_mod, dim, n):
    p = meshgen.make_problem(None, dim=dim, n=n, jitter=0.2 if dim == 2 else 0.15, seed=7, E=2.0, nu=0.35)
    p["dirichlet_dofs"] = np.zeros(0, np.int64)
    o = oracle_mod.Oracle(p, coarse_max_dofs=1)
    rp, ci, v = o.operator(0)
    A = dense_from_bsr(rp, ci, v, dim)
    assert np.array_equal(A, A.T), "assembled matrix must be bitwise symmetric"
    scale = np.abs(A).max()
    modes = rigid_modes(p["coords"])
    assert len(modes) == (3 if dim == 2 else 6)
    for t in modes:
        r = A @ t
        assert np.abs(r).max() <= 1e-12 * scale * np.abs(t).max()
    # and nothing else: the null space has exactly that dimension
    w = np.linalg.eigvalsh(A)
    assert np.sum(np.abs(w) < 1e-10 * w.max()) == len(modes)


@pytest.mark.parametrize("dim,n", [(2, 8), (3, 4)])
def test_total_load_equals_force_times_measure(oracle_mod, dim, n):
    p = meshgen.make_problem(None, dim=dim, n=n, seed=2)
    o = oracle_mod.Oracle(p)
    f = np.array([0.3, -1.7, 0.9][:dim])
    F = o.assemble_load(f).reshape(-1, dim)
    # the mesh covers the unit square / cube exactly
    np.testing.assert_allclose(F.sum(axis=0), f * 1.0, rtol=1e-12)
    np.testing.assert_allclose(o.volumes().sum(), 1.0, rtol=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_single_element_load_closed_form(oracle_mod, dim, seed):
    """F_i = int_K f phi_i = f |K| / (d+1) for each vertex of one simplex (the
    integral of a P1 hat function over its element is |K|/(d+1)); |K| from the
    determinant, computed here."""
    p = _single_element(dim, seed)
    o = oracle_mod.Oracle(p, coarse_max_dofs=100)
    f = meshgen.Stream(40 + seed).uniform(dim, -2.0, 2.0)
    F = o.assemble_load(f).reshape(dim + 1, dim)
    X = p["coords"]
    meas = abs(np.linalg.det((X[1:] - X[0]).T)) / (2.0 if dim == 2 else 6.0)
    np.testing.assert_allclose(F, np.tile(f * meas / (dim + 1), (dim + 1, 1)), rtol=1e-14, atol=0)


@pytest.mark.parametrize("dim,n,graded", [(2, 11, None), (2, 9, 8.0), (3, 6, None), (3, 7, 4.0)])
def test_load_first_moment_identity(oracle_mod, dim, n, graded):
    """P1 hat functions reproduce linear fields, sum_i phi_i(x) x_i = x, so the
    consistent load of a constant force satisfies sum_i F_i x_i^T =
    f int_Omega x^T dx exactly.  On the unit square / cube (which the jittered
    and graded meshes cover exactly) int x_b dx = 1/2 for every axis b.  A load
    put on the wrong vertex of an element changes this moment."""
    p = meshgen.make_problem(None, dim=dim, n=n, jitter=0.0 if graded else (0.2 if dim == 2 else 0.15), seed=8,
                             graded=graded)
    o = oracle_mod.Oracle(p)
    f = np.array([0.7, -1.3, 0.4][:dim])
    F = o.assemble_load(f).reshape(-1, dim)
    X = p["coords"]
    moment = F.T @ X          # [a, b] = sum_i F_{i,a} x_{i,b}
    np.testing.assert_allclose(moment, np.outer(f, np.full(dim, 0.5)), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("dim,n", [(2, 10), (3, 6)])
def test_linear_displacement_patch_test(oracle_mod, dim, n):
    """Dirichlet data = a linear field on the whole boundary, f = 0: the
    discrete solution reproduces the field at every vertex."""
    p = meshgen.make_problem(None, dim=dim, n=n, jitter=0.2 if dim == 2 else 0.15, seed=11, E=5.0, nu=0.4)
    X = p["coords"]
    rs = meshgen.Stream(99)
    c0 = rs.uniform(dim, -1, 1)
    B = rs.uniform(dim * dim, -1, 1).reshape(dim, dim)
    u = c0[None, :] + X @ B.T
    bnd = np.nonzero(np.any((X == 0.0) | (X == 1.0), axis=1))[0]
    dofs = (bnd[:, None] * dim + np.arange(dim)).ravel().astype(np.int64)
    p["dirichlet_dofs"] = dofs
    p["dirichlet_values"] = u.ravel()[dofs]
    o = oracle_mod.Oracle(p)
    U, it, rr, st, _ = o.solve(np.zeros(X.shape[0] * dim), tol=1e-13, max_iters=500)
    assert st == 0
    np.testing.assert_allclose(U, u.ravel(), rtol=0, atol=1e-10 * np.abs(u).max())


@pytest.mark.parametrize("dim,n,seed", [(2, 17, 5), (3, 6, 6)])
def test_fine_only_setup_agrees_with_full_setup(oracle_mod, dim, n, seed):
    """The assembly-only oracle (used at full sizes) gives the operator, load,
    keys and sorted-key leaves of the full setup, bit for bit."""
    p = meshgen.make_problem(None, dim=dim, n=n, jitter=0.2, seed=seed)
    full = oracle_mod.Oracle(p)
    fine = oracle_mod.Oracle(p, fine_only=True)
    x = meshgen.Stream(seed).uniform(full.n, -1.0, 1.0)
    assert np.array_equal(full.apply_A(0, x), fine.apply_A(0, x))
    assert np.array_equal(full.assemble_load(p["body_force"]), fine.assemble_load(p["body_force"]))
    assert np.array_equal(full.morton(), fine.morton())
    assert np.array_equal(full.box(), fine.box())
    assert np.array_equal(full.leaves(), fine.leaves(True))
