"""Full-size workloads, in the configuration bench.py times.

The oracle's full setup is too slow at these sizes, so the GPU path is checked
against the oracle's fine level (assembly, keys, sorted-key leaves) and
against properties that hold at any size:

  * bounding square, Morton keys and leaves bit-exact with the oracle;
  * every colouring proper and greedy by priority (fine level: splitmix64 of
    the vertex; coarse levels: lattice class first);
  * interpolation rows: partition of unity, weights in [0, 1], exact
    reproduction of the linear coordinate fields (bilinear / trilinear);
  * the solve: the true FP64 residual ||F - A U|| / ||F||, with A and F
    assembled by the oracle, is below the tolerance and equals the residual
    the solver reports.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2505_09064_gb300 import meshgen, vasmg  # noqa: E402
from tests.helpers import K_of, deinterleave  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def built():
    import __graft_entry__

    __graft_entry__.build()
    oracle.build()
    torch.cuda.set_device(0)
    return True


def _priority(s, l, nv, dim):
    sm = meshgen.splitmix64(np.arange(nv, dtype=np.uint64))
    if l == 0:
        return sm
    K = K_of(dim)
    D = int(s.export(vasmg.EXPORT_CELLS, l, np.int64).reshape(-1, 2)[:, 0].max())
    q = deinterleave(s.export(vasmg.EXPORT_LATTICE, l, np.uint64), dim, K + 1) >> np.uint64(K - D)
    cls = np.zeros(nv, dtype=np.uint64)
    w = 1
    for a in range(dim):
        cls += (q[:, a] % np.uint64(3)) * np.uint64(w)
        w *= 3
    return ((np.uint64(w - 1) - cls) << np.uint64(58)) | (sm >> np.uint64(6))


def _check_colouring(rp, ci, colour, prio):
    """Proper, and each vertex takes the smallest colour unused by its
    neighbours of higher priority (ties: smaller vertex first)."""
    nv = colour.size
    rows = np.repeat(np.arange(nv, dtype=np.int64), np.diff(rp))
    off = rows != ci
    i, j = rows[off], ci[off].astype(np.int64)
    assert np.all(colour[i] != colour[j])
    higher = (prio[j] > prio[i]) | ((prio[j] == prio[i]) & (j < i))
    ncol = int(colour.max()) + 1
    used = np.zeros((nv, ncol + 1), dtype=bool)
    used[i[higher], colour[j[higher]]] = True
    mex = np.argmin(used, axis=1)
    assert np.array_equal(mex, colour)


def _check_interpolation(s, l, dim, fine_coords):
    """Rows of P_l: partition of unity, weights in [0,1], exact reproduction of
    the coordinate fields given the coarse lattice points."""
    K = K_of(dim)
    rp = s.export(vasmg.EXPORT_P_RP, l, np.int64)
    ci = s.export(vasmg.EXPORT_P_CI, l, np.int32)
    w = s.export(vasmg.EXPORT_P_W, l, np.float64)
    rows = np.repeat(np.arange(rp.size - 1), np.diff(rp))
    assert np.all(w >= 0.0) and np.all(w <= 1.0)
    np.testing.assert_allclose(np.bincount(rows, weights=w, minlength=rp.size - 1), 1.0, rtol=0, atol=1e-12)
    coarse = deinterleave(s.export(vasmg.EXPORT_LATTICE, l + 1, np.uint64), dim, K + 1).astype(np.float64) / 2.0**K
    for a in range(dim):
        rec = np.bincount(rows, weights=w * coarse[ci, a], minlength=rp.size - 1)
        np.testing.assert_allclose(rec, fine_coords[:, a], rtol=0, atol=1e-12)


def _normalised(prob, box):
    m, M = box
    return (np.asarray(prob["coords"], dtype=np.float64) - m) / (M - m)


CASES = [
    ("square1024_checker", "fp32", 4),
    ("square1024_checker", "fp64", 4),
    ("cube64", "fp32", 3),
    ("cube128_graded", "bf16", 1),
]


@pytest.mark.parametrize("name,precision,check_levels", CASES)
def test_full_size_workload(built, name, precision, check_levels):
    prob = meshgen.make_problem(name)
    dim = prob["dim"]
    o = oracle.Oracle(prob, fine_only=True)
    s = vasmg.Solver(prob, precision=precision, stream=torch.cuda.current_stream().cuda_stream)
    try:
        box = s.export(vasmg.EXPORT_BOX, 0, np.float64)
        assert np.array_equal(box, o.box())
        assert np.array_equal(s.export(vasmg.EXPORT_MORTON, 0, np.uint64), o.morton())
        assert np.array_equal(s.export(vasmg.EXPORT_LEAF, 0, np.int64).reshape(-1, 2), o.leaves(True))
        L = s.num_levels
        # colourings and interpolation on the first levels (the coarse ones are
        # covered at small sizes by the bit-exact parity tests)
        for l in range(min(check_levels, L - 1)):
            nv = s.level_info(l)[0]
            rp = s.export(vasmg.EXPORT_A_RP, l, np.int64)
            ci = s.export(vasmg.EXPORT_A_CI, l, np.int32)
            _check_colouring(rp, ci, s.export(vasmg.EXPORT_COLOUR, l, np.int32), _priority(s, l, nv, dim))
            if l == 0:
                fine = _normalised(prob, box)
            else:
                fine = deinterleave(s.export(vasmg.EXPORT_LATTICE, l, np.uint64), dim,
                                    K_of(dim) + 1).astype(np.float64) / 2.0**K_of(dim)
            _check_interpolation(s, l, dim, fine)
        # the solve, checked by the oracle's FP64 operator
        F = o.assemble_load(prob["body_force"])
        F[prob["dirichlet_dofs"]] = 0.0
        Fd = torch.tensor(F, dtype=torch.float64, device="cuda")
        Ud = torch.zeros_like(Fd)
        rc, st, _ = s.solve(Fd, Ud, 1e-6)
        assert rc == 0 and 0 < st.iterations < 200
        U = Ud.cpu().numpy()
        r = F - o.apply_A(0, U)
        true_rel = float(np.linalg.norm(r) / np.linalg.norm(F))
        assert true_rel < 1e-6 * (1 + 1e-6)
        assert abs(true_rel - st.rel_res) <= 1e-9
    finally:
        s.close()


@pytest.mark.parametrize("dim,n", [(2, 300), (3, 32)])
def test_galerkin_levels_keep_rigid_modes_large(built, dim, n):
    """At sizes the full oracle does not reach: without Dirichlet data every
    Galerkin level the device builds annihilates the rigid-body modes at its
    own vertices (P reproduces linear fields, A_0 annihilates them) -- on its
    live rows.  A coarse dof that no fine dof interpolates from with a
    nonzero weight is dead and carries an identity row, which the rigid modes
    are not in the kernel of."""
    import scipy.sparse as sp
    from scipy.sparse.linalg import norm as sparse_norm

    from tests.helpers import rigid_modes

    prob = meshgen.make_problem(None, dim=dim, n=n, jitter=0.2 if dim == 2 else 0.15, seed=90 + n)
    prob["dirichlet_dofs"] = np.zeros(0, dtype=np.int64)
    prob.pop("dirichlet_values", None)
    s = vasmg.Solver(prob, precision="fp64", stream=torch.cuda.current_stream().cuda_stream)
    try:
        box = s.export(vasmg.EXPORT_BOX, 0, np.float64)
        K = K_of(dim)
        assert s.num_levels >= 4
        for l in range(s.num_levels):
            rp = s.export(vasmg.EXPORT_A_RP, l, np.int64)
            ci = s.export(vasmg.EXPORT_A_CI, l, np.int32)
            v = s.export(vasmg.EXPORT_A_V, l, np.float64).reshape(-1, dim, dim)
            A = sp.bsr_matrix((v, ci, rp), shape=((rp.size - 1) * dim, (rp.size - 1) * dim)).tocsr()
            if l == 0:
                X = np.asarray(prob["coords"], dtype=np.float64)
            else:
                q = deinterleave(s.export(vasmg.EXPORT_LATTICE, l, np.uint64), dim, K + 1).astype(np.float64)
                X = box[0] + (box[1] - box[0]) * q / 2.0 ** K
            scale = sparse_norm(A)
            live = ~s.export(vasmg.EXPORT_DEAD, l, np.uint8).astype(bool)
            for t in rigid_modes(X):
                r = np.linalg.norm((A @ t)[live]) / (scale * np.linalg.norm(t))
                assert r <= 1e-12, (l, r)
    finally:
        s.close()
