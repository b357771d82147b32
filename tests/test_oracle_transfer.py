"""Pins for the oracle's coarse grids, interpolation weights (Sec. 3.2) and
Galerkin operators (eq. (Ac)): partition of unity, exact reproduction of
bilinear / trilinear fields, weights in [0,1], Theorem 3.2 (threshold 9 on a
uniform grid gives textbook geometric multigrid), and P^T A P against a dense
numpy product."""
import os

import numpy as np
import pytest

from paper_2505_09064_gb300 import meshgen
from tests.helpers import K_of, deinterleave, dense_from_bsr, dense_P

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _prob(dim, n, seed):
    return meshgen.make_problem(None, dim=dim, n=n, seed=seed, jitter=0.2 if dim == 2 else 0.15)


def _level_coords(o, l, dim):
    """Physical coordinates of the vertices of level l (fine: the mesh)."""
    if l == 0:
        return o.coords
    m, M = o.box()
    K = K_of(dim)
    p = deinterleave(o.lattice(l), dim, K + 1).astype(np.float64)
    return m + (M - m) * p / 2.0 ** K


def _multilinear_fields(X):
    d = X.shape[1]
    fields = [np.ones(len(X))] + [X[:, a] for a in range(d)]
    fields.append(X[:, 0] * X[:, 1])
    if d == 3:
        fields += [X[:, 1] * X[:, 2], X[:, 0] * X[:, 2], X[:, 0] * X[:, 1] * X[:, 2]]
    return fields


@pytest.mark.parametrize("dim,n,seed", [(2, 14, 1), (2, 23, 4), (3, 6, 2), (3, 7, 5)])
def test_weights_partition_of_unity_and_reproduction(oracle_mod, dim, n, seed):
    p = _prob(dim, n, seed)
    p["coords"] = p["coords"] * 2.0 + 1.0  # non-unit box
    o = oracle_mod.Oracle(p)
    for l in range(o.num_levels - 1):
        rp, ci, w = o.prolongation(l)
        assert np.all(w > 0) and np.all(w <= 1)
        sums = np.add.reduceat(w, rp[:-1])
        np.testing.assert_allclose(sums, 1.0, rtol=0, atol=1e-14)
        Xf = _level_coords(o, l, dim)
        Xc = _level_coords(o, l + 1, dim)
        nf = len(rp) - 1
        rows = np.repeat(np.arange(nf), np.diff(rp))
        for g_f, g_c in zip(_multilinear_fields(Xf), _multilinear_fields(Xc)):
            interp = np.zeros(nf)
            np.add.at(interp, rows, w * g_c[ci])
            np.testing.assert_allclose(interp, g_f, rtol=0, atol=1e-12 * max(1.0, np.abs(g_f).max()))


def test_coincident_vertex_gets_weight_one(oracle_mod):
    p = _prob(2, 9, 3)
    o = oracle_mod.Oracle(p)
    rp, ci, w = o.prolongation(0)
    # the four corners of the unit square coincide with lattice corners of the root
    X = p["coords"]
    for v in np.nonzero(np.all((X == 0) | (X == 1), axis=1))[0]:
        assert rp[v + 1] - rp[v] == 1 and w[rp[v]] == 1.0


def _textbook_P1d(m):
    """1D linear interpolation from m+1 coarse to 2m+1 fine points."""
    P = np.zeros((2 * m + 1, m + 1))
    for i in range(m + 1):
        P[2 * i, i] = 1.0
    for i in range(m):
        P[2 * i + 1, i] = 0.5
        P[2 * i + 1, i + 1] = 0.5
    return P


@pytest.mark.parametrize("dim,k", [(2, 2), (2, 4), (3, 2), (3, 3)])
def test_theorem_3_2_threshold_9_is_textbook_gmg(oracle_mod, dim, k):
    """With the leaf capacity set to 9 (27 in 3D) a uniform (2^k+1)^d grid gives
    every level = textbook bilinear (trilinear) interpolation with coarsening
    by two (Theorem 3.2)."""
    n = 2 ** k + 1
    p = meshgen.make_problem(None, dim=dim, n=n, jitter=0.0, seed=1)
    o = oracle_mod.Oracle(p, threshold=9 if dim == 2 else 27)
    K = K_of(dim)
    assert o.num_levels == k + 1
    for l in range(o.num_levels - 1):
        mf, mc = 2 ** (k - l), 2 ** (k - l - 1)
        P1 = _textbook_P1d(mc)
        Pref = P1
        for _ in range(dim - 1):
            Pref = np.kron(P1, Pref)  # row-major: x fastest
        # map oracle vertex order to grid order
        def grid_index(lv, m):
            if lv == 0:
                return np.arange(n ** dim)
            c = deinterleave(o.lattice(lv), dim, K + 1).astype(np.int64) // (2 ** K // m)
            idx = np.zeros(len(c), dtype=np.int64)
            for a in reversed(range(dim)):
                idx = idx * (m + 1) + c[:, a]
            return idx
        gf, gc = grid_index(l, mf), grid_index(l + 1, mc)
        rp, ci, w = o.prolongation(l)
        P = np.zeros(((mf + 1) ** dim, (mc + 1) ** dim))
        for i in range(len(rp) - 1):
            for kk in range(rp[i], rp[i + 1]):
                P[gf[i], gc[ci[kk]]] = w[kk]
        np.testing.assert_array_equal(P, Pref)


def test_theorem_3_2_golden_stencil(oracle_mod):
    """Golden fixture: the column of the centre coarse vertex of a 5x5 uniform
    grid with leaf capacity 9 is the classical 3x3 stencil (Theorem 3.2)."""
    ref = np.loadtxt(os.path.join(GOLDEN, "thm32_centre_column_5x5.txt"))
    p = meshgen.make_problem(None, dim=2, n=5, jitter=0.0, seed=1)
    o = oracle_mod.Oracle(p, threshold=9)
    rp, ci, w = o.prolongation(0)
    c = deinterleave(o.lattice(1), 2, 32).astype(np.int64) // 2 ** 30
    centre = int(np.nonzero((c[:, 0] == 1) & (c[:, 1] == 1))[0][0])
    col = np.zeros(25)
    for i in range(25):
        for kk in range(rp[i], rp[i + 1]):
            if ci[kk] == centre:
                col[i] = w[kk]
    np.testing.assert_array_equal(col.reshape(5, 5), ref)


@pytest.mark.parametrize("dim,n,seed", [(2, 7, 1), (2, 9, 6), (3, 4, 2)])
def test_galerkin_equals_dense_product(oracle_mod, dim, n, seed):
    p = _prob(dim, n, seed)
    o = oracle_mod.Oracle(p)
    for l in range(min(o.num_levels - 1, 3)):
        rp, ci, v = o.operator(l)
        A = dense_from_bsr(rp, ci, v, dim)
        prp, pci, pw = o.prolongation(l)
        nc = o.nv_level(l + 1)
        dead_f = o.dead(l)
        P = dense_P(prp, pci, pw, nc, dim, dead_f)
        Ac_ref = P.T @ A @ P
        dead_c = o.dead(l + 1)
        # dead coarse dofs: empty masked column -> identity row
        assert np.array_equal(dead_c.astype(bool), ~np.any(P != 0, axis=0))
        for i in np.nonzero(dead_c)[0]:
            Ac_ref[i, i] = 1.0
        crp, cci, cv = o.operator(l + 1)
        Ac = dense_from_bsr(crp, cci, cv, dim)
        np.testing.assert_allclose(Ac, Ac_ref, rtol=0, atol=1e-12 * np.abs(Ac_ref).max())
        assert np.array_equal(Ac, Ac.T) or np.abs(Ac - Ac.T).max() <= 1e-13 * np.abs(Ac).max()


def test_level_count_merges_to_root(oracle_mod):
    p = _prob(2, 33, 2)
    o = oracle_mod.Oracle(p)
    L = o.num_levels
    assert o.nv_level(L - 1) == 4
    depths = [int(o.cells(l)[:, 0].max()) for l in range(1, L)]
    # each merge removes exactly the deepest layer (Sec. 3.1.2)
    assert depths == list(range(depths[0], -1, -1))


@pytest.mark.parametrize("dim,n,seed", [(2, 14, 7), (2, 19, 9), (3, 6, 8)])
def test_coarse_levels_keep_the_rigid_body_modes(oracle_mod, dim, n, seed):
    """Without Dirichlet data A_0 annihilates the rigid-body modes, and P
    reproduces linear fields exactly, so every Galerkin level
    A_{l+1} = P^T A_l P annihilates the rigid modes evaluated at its own
    vertices (translations and rotations are linear in the coordinates) on
    its live rows; a dead coarse dof (no fine dof interpolates from it with a
    nonzero weight) carries an identity row instead."""
    from tests.helpers import rigid_modes

    p = _prob(dim, n, seed)
    p["dirichlet_dofs"] = np.zeros(0, dtype=np.int64)
    p.pop("dirichlet_values", None)
    o = oracle_mod.Oracle(p)
    assert o.num_levels >= 3
    for l in range(o.num_levels):
        rp, ci, v = o.operator(l)
        A = dense_from_bsr(rp, ci, v, dim)
        live = ~o.dead(l).astype(bool)
        X = _level_coords(o, l, dim)
        for t in rigid_modes(X):
            r = np.linalg.norm((A @ t)[live]) / (np.linalg.norm(A) * np.linalg.norm(t))
            assert r <= 1e-12, (l, r)
