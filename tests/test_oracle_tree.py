"""Pins for the oracle's auxiliary region tree (Sec. 3.1.1): bounding square,
quantisation, insertion-order invariance of the point-region tree, the split
rule checked by brute-force counting, and the depth bound of Theorem 3.1."""
import itertools

import numpy as np
import pytest

from paper_2505_09064_gb300 import meshgen
from tests.helpers import K_of


def _prob(dim, n, seed, jitter=None):
    return meshgen.make_problem(None, dim=dim, n=n, seed=seed,
                                jitter=(0.2 if dim == 2 else 0.15) if jitter is None else jitter)


@pytest.mark.parametrize("dim,n", [(2, 12), (3, 6)])
def test_bounding_square_and_keys_brute_force(oracle_mod, dim, n):
    p = _prob(dim, n, 3)
    X = p["coords"] * 3.0 - 0.5  # move away from the unit box
    X[:, 0] *= 0.5                # and make it non-square
    p["coords"] = X
    o = oracle_mod.Oracle(p)
    m, M = o.box()
    assert m == X.min() and M == X.max()
    K = K_of(dim)
    keys = o.morton()
    # brute force: quantise with python integers, interleave bit by bit
    for v in range(0, X.shape[0], 7):
        q = []
        for a in range(dim):
            t = (X[v, a] - m) / (M - m)
            q.append(min(int(np.floor(t * 2.0 ** K)), 2 ** K - 1))
        key = 0
        for b in range(K):
            for a in range(dim):
                key |= ((q[a] >> b) & 1) << (b * dim + a)
        assert int(keys[v]) == key


def _count_in_cell(keys_sorted, key, depth, dim, K):
    rest = dim * (K - depth)
    lo = (key >> rest) << rest
    hi = lo + (1 << rest)
    return np.searchsorted(keys_sorted, np.uint64(lo), "left") - (
        np.searchsorted(keys_sorted, np.uint64(hi), "left") if hi < 2 ** 64 else len(keys_sorted))


@pytest.mark.parametrize("dim,n,T", [(2, 11, 4), (2, 9, 9), (3, 5, 8), (3, 6, 4)])
def test_split_rule_by_counting(oracle_mod, dim, n, T):
    """Each vertex's leaf holds <= T vertices and its parent holds > T
    (split iff the vertex set exceeds the threshold, Step 2)."""
    p = _prob(dim, n, 5)
    o = oracle_mod.Oracle(p, threshold=T)
    K = K_of(dim)
    keys = o.morton().astype(np.uint64)
    ks = np.sort(keys)
    leaves = o.leaves()
    for v in range(len(keys)):
        depth, ck = int(leaves[v, 0]), int(leaves[v, 1])
        assert ck == int(keys[v]) >> (dim * (K - depth))
        cnt = -_count_in_cell(ks, int(keys[v]), depth, dim, K)
        assert 1 <= cnt <= T or depth == K
        if depth > 0:
            parent = -_count_in_cell(ks, int(keys[v]), depth - 1, dim, K)
            assert parent > T


@pytest.mark.parametrize("dim,n", [(2, 13), (3, 6)])
def test_insertion_order_invariance(oracle_mod, dim, n):
    """The tree from sequential insertion does not depend on the order in which
    vertices are inserted, and equals the sort/count construction."""
    p = _prob(dim, n, 8)
    base = oracle_mod.Oracle(p).leaves()
    sorted_build = oracle_mod.Oracle(p).leaves(sorted_method=True)
    assert np.array_equal(base, sorted_build)
    nv = p["coords"].shape[0]
    for s in range(3):
        perm = np.argsort(meshgen.Stream(40 + s).u64(nv)).astype(np.int64)
        lv = oracle_mod.Oracle(p, insertion_order=perm).leaves()
        assert np.array_equal(base, lv)


def test_literal_insertion_small_example(oracle_mod):
    """Five points in the unit square with T = 4 (Step 2.2): the fifth insertion
    splits the root; all points land in depth-1 cells except where a quadrant
    receives more than four."""
    pts = np.array([[0.1, 0.1], [0.9, 0.1], [0.1, 0.9], [0.9, 0.9], [0.6, 0.7],
                    [0.0, 0.0], [1.0, 1.0]])
    elems = np.array([[0, 1, 4], [0, 4, 2], [1, 3, 4], [4, 3, 2], [5, 1, 0], [3, 6, 2]], dtype=np.int32)
    p = dict(dim=2, coords=pts, elems=elems, lam=np.ones(6), mu=np.ones(6),
             dirichlet_dofs=np.zeros(0, np.int64), dirichlet_values=None)
    o = oracle_mod.Oracle(p, threshold=4)
    lv = o.leaves()
    # 7 points > 4 -> root split; quadrants: SW {0,5}, SE {1}, NW {2}, NE {3,4,6}
    assert np.all(lv[:, 0] == 1)
    quadrant = lambda x, y: (1 if x >= 0.5 else 0) | ((1 if y >= 0.5 else 0) << 1)
    for v, (x, y) in enumerate(pts):
        assert lv[v, 1] == quadrant(x, y)


@pytest.mark.parametrize("dim,n,seed", [(2, 12, 1), (2, 20, 2), (3, 6, 3), (3, 8, 4)])
def test_depth_bound_theorem_3_1(oracle_mod, dim, n, seed):
    """Theorem 3.1: depth <= log2(d_max/d_min) + 3/2 in 2D (root = depth 1);
    in 3D diam(D^1) <= sqrt(3) d_max gives log2(d_max/d_min) + log2(sqrt 3) + 1.
    One level of slack: a leaf's *parent* is what holds two distinct points."""
    p = _prob(dim, n, seed)
    X = p["coords"]
    o = oracle_mod.Oracle(p)
    D = np.sqrt(((X[:, None, :] - X[None, :, :]) ** 2).sum(-1))
    dmax = D.max()
    dmin = D[D > 0].min()
    bound = np.log2(dmax / dmin) + (1.5 if dim == 2 else np.log2(np.sqrt(3)) + 1)
    depth_paper = o.leaves()[:, 0].max() + 1
    assert depth_paper <= bound + 1


def test_every_vertex_in_exactly_one_leaf_and_leaves_disjoint(oracle_mod):
    p = _prob(2, 17, 9)
    o = oracle_mod.Oracle(p)
    cells = o.cells(1)
    K = 31
    # cells of level 1 are the distinct non-empty leaves and cover disjoint key ranges
    lv = o.leaves()
    distinct = {tuple(r) for r in lv.tolist()}
    assert distinct == {tuple(r) for r in cells.tolist()}
    ranges = sorted(((int(k) << (2 * (K - int(dp)))), (int(k) + 1) << (2 * (K - int(dp)))) for dp, k in cells)
    for (a0, a1), (b0, b1) in itertools.pairwise(ranges):
        assert a1 <= b0
