"""Pins for the oracle's cycle variants: the W-cycle (Fig. 2) and the additive
form B_h = S_h + Pi B_0 Pi^T (Sec. 4), beside the V-cycle (Alg. 3).

Every operator is rebuilt densely from the exported levels (A_l, P_l with the
dead-dof masks, colours) in the textbook matrix form of multigrid, with no
call into the oracle's smoother or cycle:

* a forward multicolour block GS sweep from x is x + (D + L)^{-1} (b - A x),
  L the blocks whose column has an earlier colour; the backward sweep uses
  D + U with U the later-colour blocks;
* a cycle with gamma coarse corrections on level l, applied to b from zero,
  is x1 = M_f b, x2 = x1 + P C P^T (b - A x1), x = x2 + M_b (b - A x2) with
  M_f = (D + L)^{-1}, M_b = (D + U)^{-1} and C = sum_{k < g} (I - B_c A_c)^k
  B_c, i.e. g cycles on the coarse problem from zero (g = 1 when level l+1 is
  the coarsest, solved exactly).  So B_l = M_b + (I - M_b A)(M_f + P C P^T
  (I - A M_f)); no inverse of an A_l is formed except on the coarsest level,
  since the coarse operators of these meshes can be badly conditioned;
* the additive form is SGS(r) + P_0 B_1 P_0^T r, SGS the forward-then-
  backward sweep pair from zero.

The oracle's preconditioner, applied to unit vectors, must equal these
matrices; both must be symmetric positive definite, and PCG must converge
with each.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_2505_09064_gb300 import meshgen
from tests.helpers import dense_P, dense_from_bsr


def _prob(dim, n, seed, **kw):
    return meshgen.make_problem(None, dim=dim, n=n, seed=seed, jitter=0.2 if dim == 2 else 0.15, **kw)


def _levels(o, dim):
    """Dense A_l, masked P_l, and the sweep splittings D + L, D + U per level."""
    L = o.num_levels
    out = []
    for l in range(L):
        rp, ci, v = o.operator(l)
        A = dense_from_bsr(rp, ci, v, dim)
        lev = {"A": A}
        if l + 1 < L:
            colour = np.repeat(o.colours(l), dim)
            earlier = colour[None, :] < colour[:, None]
            later = colour[None, :] > colour[:, None]
            same = colour[None, :] == colour[:, None]
            lev["DL"] = np.where(earlier | same, A, 0.0)
            lev["DU"] = np.where(later | same, A, 0.0)
            prp, pci, pw = o.prolongation(l)
            nc = o.level_info(l + 1)[0]
            lev["P"] = dense_P(prp, pci, pw, nc, dim, dead_fine=o.dead(l))
        out.append(lev)
    return out


def _cycle(levels, l, gamma):
    """Dense B_l of the gamma-cycle from level l (exact inverse on the coarsest)."""
    A = levels[l]["A"]
    if l + 1 == len(levels):
        return np.linalg.inv(A)
    n = A.shape[0]
    I = np.eye(n)
    Ac = levels[l + 1]["A"]
    Bc = _cycle(levels, l + 1, gamma)
    g = 1 if l + 2 == len(levels) else gamma
    Ec = np.eye(Ac.shape[0]) - Bc @ Ac
    C = sum(np.linalg.matrix_power(Ec, k) for k in range(g)) @ Bc
    P = levels[l]["P"]
    Mf = np.linalg.solve(levels[l]["DL"], I)
    Mb = np.linalg.solve(levels[l]["DU"], I)
    G = Mf + P @ C @ P.T @ (I - A @ Mf)
    return Mb + (I - Mb @ A) @ G


def _additive(levels, gamma):
    A = levels[0]["A"]
    I = np.eye(A.shape[0])
    Mf = np.linalg.solve(levels[0]["DL"], I)
    Mb = np.linalg.solve(levels[0]["DU"], I)
    sgs = Mf + Mb - Mb @ A @ Mf
    P = levels[0]["P"]
    B1 = _cycle(levels, 1, gamma)
    return sgs + P @ B1 @ P.T


def _oracle_matrix(o, n):
    return np.stack([o.precondition(e) for e in np.eye(n)], axis=1)


CASES = [
    # (dim, n, seed, coarse_max_dofs): hierarchies of 4+ levels, so that the
    # W-cycle differs from the V-cycle on at least two levels
    (2, 9, 41, 0),
    (2, 11, 42, 0),
    (3, 5, 43, 0),
]


@pytest.mark.parametrize("dim,n,seed,cmax", CASES)
def test_v_and_w_cycles_equal_dense_multigrid(oracle_mod, dim, n, seed, cmax):
    p = _prob(dim, n, seed, nu=0.35)
    o = oracle_mod.Oracle(p, coarse_max_dofs=cmax)
    assert o.num_levels >= 4
    lev = _levels(o, dim)
    N = lev[0]["A"].shape[0]
    for gamma in (1, 2, 3):
        o.set_cycle(gamma=gamma)
        B = _oracle_matrix(o, N)
        Bd = _cycle(lev, 0, gamma)
        scale = np.abs(Bd).max()
        assert np.abs(B - Bd).max() <= 1e-10 * scale, gamma
        assert np.abs(B - B.T).max() <= 1e-11 * scale
        assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0
    # the W-cycle is a different operator from the V-cycle here
    o.set_cycle(gamma=1)
    BV = _oracle_matrix(o, N)
    o.set_cycle(gamma=2)
    BW = _oracle_matrix(o, N)
    assert np.abs(BV - BW).max() > 1e-6 * np.abs(BV).max()


@pytest.mark.parametrize("dim,n,seed,cmax", CASES + [(2, 10, 44, 60)])
def test_additive_form_equals_dense(oracle_mod, dim, n, seed, cmax):
    p = _prob(dim, n, seed, nu=0.3)
    o = oracle_mod.Oracle(p, coarse_max_dofs=cmax)
    lev = _levels(o, dim)
    N = lev[0]["A"].shape[0]
    for gamma in (1, 2):
        o.set_cycle(gamma=gamma, additive=True)
        B = _oracle_matrix(o, N)
        Bd = _additive(lev, gamma)
        scale = np.abs(Bd).max()
        assert np.abs(B - Bd).max() <= 1e-10 * scale
        assert np.abs(B - B.T).max() <= 1e-11 * scale
        assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0


def test_additive_two_level_uses_the_exact_coarse_inverse(oracle_mod):
    """With level 1 the coarsest, B_0 = A_1^{-1}: the paper's choice."""
    p = _prob(2, 10, 45)
    o = oracle_mod.Oracle(p, coarse_max_dofs=160)  # 200 fine dofs, 146 on level 1
    assert o.num_levels == 2
    lev = _levels(o, 2)
    N = lev[0]["A"].shape[0]
    o.set_cycle(additive=True)
    B = _oracle_matrix(o, N)
    A = lev[0]["A"]
    P = lev[0]["P"]
    I = np.eye(N)
    Mf = np.linalg.solve(lev[0]["DL"], I)
    Mb = np.linalg.solve(lev[0]["DU"], I)
    Bd = Mf + Mb - Mb @ A @ Mf + P @ np.linalg.inv(lev[1]["A"]) @ P.T
    assert np.abs(B - Bd).max() <= 1e-10 * np.abs(Bd).max()


@pytest.mark.parametrize("dim,n,seed", [(2, 33, 46), (3, 9, 47)])
def test_pcg_converges_with_each_variant(oracle_mod, dim, n, seed):
    p = _prob(dim, n, seed)
    o = oracle_mod.Oracle(p)
    F = o.assemble_load(p["body_force"])
    F[p["dirichlet_dofs"]] = 0.0
    its = {}
    sols = {}
    for name, kw in [("V", dict(gamma=1)), ("W", dict(gamma=2)), ("additive", dict(additive=True))]:
        o.set_cycle(**kw)
        U, it, rr, st, _ = o.solve(F, tol=1e-8)
        assert st == 0 and rr < 1e-8
        its[name] = it
        sols[name] = U
    # same solution to the tolerance; the W-cycle needs no more iterations
    # than the V-cycle, the additive form (a weaker preconditioner) no fewer
    for name in ("W", "additive"):
        assert np.abs(sols[name] - sols["V"]).max() <= 1e-6 * np.abs(sols["V"]).max()
    assert its["W"] <= its["V"]
    assert its["additive"] >= its["V"]
