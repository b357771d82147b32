"""Parity of the CUDA library (through the C ABI) with the CPU FP64 oracle.

Integer and geometric work must match bit for bit: Morton keys, leaves, cells,
lattice vertices, interpolation patterns *and weights*, operator patterns,
dead dofs and colours.  Floating-point results are compared element by
element: every entry's error relative to the largest entry of the reference
(max norm).  FP64 values match to 1e-12; a full FP64 solve matches the
oracle's solution to 1e-10 with the same iteration count (+-1).  Mixed
precision solves must reach a true relative residual below the tolerance
(1e-6); their error against the FP64 oracle is reported.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2505_09064_gb300 import meshgen, vasmg  # noqa: E402

pytestmark = pytest.mark.gpu

CASES = {
    "2d_n24": dict(dim=2, n=24, jitter=0.2, seed=1),
    "2d_n37_ragged": dict(dim=2, n=37, jitter=0.2, seed=7, E=3.0, nu=0.4),
    "3d_n8": dict(dim=3, n=8, jitter=0.15, seed=3),
    "3d_n11_graded": dict(dim=3, n=11, jitter=0.0, seed=4, nu=0.45, graded=16.0),
}


def _prob(name):
    return meshgen.make_problem(None, **CASES[name])


@pytest.fixture(scope="module")
def built():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)
    return True


_cache = {}


def pair(name, precision="fp64", threshold=0):
    key = (name, precision, threshold)
    if key not in _cache:
        p = _prob(name)
        o = oracle.Oracle(p, threshold=threshold)
        s = vasmg.Solver(p, precision=precision, stream=torch.cuda.current_stream().cuda_stream, threshold=threshold)
        _cache[key] = (p, o, s)
    return _cache[key]


def _sorted_cells(a):
    a = a.reshape(-1, 2)
    return a[np.lexsort((a[:, 1], a[:, 0]))]


@pytest.mark.parametrize("name", list(CASES))
def test_tree_and_hierarchy_bit_exact(built, name):
    p, o, s = pair(name)
    assert s.num_levels == o.num_levels
    assert np.array_equal(s.export(vasmg.EXPORT_BOX, 0, np.float64), o.box())
    assert np.array_equal(s.export(vasmg.EXPORT_MORTON, 0, np.uint64), o.morton())
    assert np.array_equal(s.export(vasmg.EXPORT_LEAF, 0, np.int64).reshape(-1, 2), o.leaves())
    for l in range(1, o.num_levels):
        assert np.array_equal(_sorted_cells(s.export(vasmg.EXPORT_CELLS, l)), _sorted_cells(o.cells(l)))
        assert np.array_equal(s.export(vasmg.EXPORT_LATTICE, l, np.uint64), o.lattice(l))
    for l in range(o.num_levels - 1):
        orp, oci, ow = o.prolongation(l)
        assert np.array_equal(s.export(vasmg.EXPORT_P_RP, l, np.int64), orp)
        assert np.array_equal(s.export(vasmg.EXPORT_P_CI, l, np.int32), oci)
        assert np.array_equal(s.export(vasmg.EXPORT_P_W, l, np.float64), ow)  # bit-exact weights


@pytest.mark.parametrize("name", list(CASES))
def test_operators_colours_exact(built, name):
    p, o, s = pair(name)
    d = p["dim"]
    np.testing.assert_allclose(s.export(vasmg.EXPORT_VOL, 0, np.float64), o.volumes(), rtol=1e-13)
    for l in range(o.num_levels):
        orp, oci, ov = o.operator(l)
        assert np.array_equal(s.export(vasmg.EXPORT_A_RP, l, np.int64), orp)
        assert np.array_equal(s.export(vasmg.EXPORT_A_CI, l, np.int32), oci)
        sv = s.export(vasmg.EXPORT_A_V, l, np.float64).reshape(-1, d, d)
        scale = np.abs(ov).max()
        np.testing.assert_allclose(sv, ov, rtol=0, atol=1e-12 * scale)
        if l == 0:
            # exactly symmetric on the device too
            rp, ci = orp, oci
            rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
            pos = {(int(i), int(j)): k for k, (i, j) in enumerate(zip(rows, ci))}
            for k, (i, j) in enumerate(zip(rows, ci)):
                assert np.array_equal(sv[k], sv[pos[(int(j), int(i))]].T)
        assert np.array_equal(s.export(vasmg.EXPORT_DEAD, l, np.uint8), o.dead(l))
        assert np.array_equal(s.export(vasmg.EXPORT_COLOUR, l, np.int32), o.colours(l))
        np.testing.assert_allclose(s.export(vasmg.EXPORT_DINV, l, np.float64),
                                   o.export(oracle.DINV, l, np.float64), rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("name", ["2d_n24", "3d_n8"])
def test_load_vector(built, name):
    p, o, s = pair(name)
    F_ref = o.assemble_load(p["body_force"])
    F = torch.zeros(F_ref.size, dtype=torch.float64, device="cuda")
    s.assemble_load(p["body_force"], F)
    np.testing.assert_allclose(F.cpu().numpy(), F_ref, rtol=1e-13, atol=1e-16)


def _rel(a, b):
    """Element-wise error relative to the reference's largest entry (max norm)."""
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("name", ["2d_n24", "2d_n37_ragged", "3d_n8", "3d_n11_graded"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5), ("bf16", 2e-2)])
def test_single_steps(built, name, precision, tol):
    """Every row of the hot path in isolation, against the oracle's function."""
    p, o, s = pair(name, precision)
    d = p["dim"]
    rs = meshgen.Stream(77)
    L = o.num_levels
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    for l in range(L):
        nl = o.nv_level(l) * d
        dead = o.dead(l).astype(bool)
        b = rs.uniform(nl, -1, 1)
        b[dead] = 0.0
        if l == 0 and precision == "fp64":
            x = rs.uniform(nl, -1, 1)
            y = torch.zeros(nl, dtype=torch.float64, device="cuda")
            s.apply(vasmg.OP_MATVEC, 0, dev(x), y)
            assert _rel(y.cpu().numpy(), o.apply_A(0, x)) <= 1e-13
        if l == L - 1:
            y = torch.zeros(nl, dtype=torch.float64, device="cuda")
            s.apply(vasmg.OP_COARSE, l, dev(b), y)
            assert _rel(y.cpu().numpy(), o.coarse_solve(b)) <= max(tol, 1e-11)
            continue
        # forward sweep from zero
        y = torch.zeros(nl, dtype=torch.float64, device="cuda")
        s.apply(vasmg.OP_SMOOTH_FWD, l, dev(b), y)
        ref_fwd = o.gs_sweep(l, b, np.zeros(nl), forward=True)
        assert _rel(y.cpu().numpy(), ref_fwd) <= tol
        # backward sweep from an arbitrary start
        x0 = rs.uniform(nl, -1, 1)
        x0[dead] = 0.0
        y = dev(x0.copy())
        s.apply(vasmg.OP_SMOOTH_BWD, l, dev(b), y)
        assert _rel(y.cpu().numpy(), o.gs_sweep(l, b, x0, forward=False)) <= tol
        # residual after the zero-start forward sweep (upper-part form)
        y = torch.zeros(nl, dtype=torch.float64, device="cuda")
        s.apply(vasmg.OP_RESIDUAL, l, dev(b), y)
        ref_r = b - o.apply_A(l, ref_fwd)
        assert np.max(np.abs(y.cpu().numpy() - ref_r)) <= tol * 10 * np.max(np.abs(b))
        # transfers
        nc = o.nv_level(l + 1) * d
        r = rs.uniform(nl, -1, 1)
        r[dead] = 0.0
        y = torch.zeros(nc, dtype=torch.float64, device="cuda")
        s.apply(vasmg.OP_RESTRICT, l, dev(r), y)
        assert _rel(y.cpu().numpy(), o.restrict(l, r)) <= max(tol, 1e-7 if precision != "fp64" else tol)
        e = rs.uniform(nc, -1, 1)
        xin = rs.uniform(nl, -1, 1)
        y = dev(xin.copy())
        s.apply(vasmg.OP_PROLONG, l, dev(e), y)
        assert _rel(y.cpu().numpy(), o.prolong_add(l, e, xin)) <= max(tol, 1e-7 if precision != "fp64" else tol)
    # a full V-cycle from every level (the small levels run in the cluster tail kernel)
    for l in range(L):
        nl = o.nv_level(l) * d
        b = rs.uniform(nl, -1, 1)
        b[o.dead(l).astype(bool)] = 0.0
        y = torch.zeros(nl, dtype=torch.float64, device="cuda")
        s.apply(vasmg.OP_VCYCLE, l, dev(b), y)
        assert _rel(y.cpu().numpy(), o.vcycle(b, level=l)) <= max(tol * 20, 1e-11)


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_solve_matches_oracle(built, name):
    p, o, s = pair(name)
    F = o.assemble_load(p["body_force"])
    U_ref, it_ref, rr_ref, st_ref, hist_ref = o.solve(F, tol=1e-6, hist_cap=200)
    assert st_ref == 0
    Fd = torch.from_numpy(F).cuda()
    U = torch.zeros_like(Fd)
    rc, st, hist = s.solve(Fd, U, tol=1e-6, history_cap=200)
    assert rc == 0
    assert abs(st.iterations - it_ref) <= 1
    assert _rel(U.cpu().numpy(), U_ref) <= 1e-10
    k = min(len(hist), len(hist_ref))
    np.testing.assert_allclose(hist[:k], hist_ref[:k], rtol=1e-8)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_mixed_precision_solve(built, name, precision):
    p, o, s = pair(name, precision)
    F = o.assemble_load(p["body_force"])
    U_ref, it_ref, _, _, _ = o.solve(F, tol=1e-10)
    Fd = torch.from_numpy(F).cuda()
    U = torch.zeros_like(Fd)
    rc, st, _ = s.solve(Fd, U, tol=1e-6)
    assert rc == 0 and st.rel_res < 1e-6
    # true residual of the returned solution, computed by the oracle's operator
    Uh = U.cpu().numpy()
    Fr = F.copy()
    Fr[p["dirichlet_dofs"]] = 0.0
    res = np.linalg.norm(Fr - o.apply_A(0, Uh)) / np.linalg.norm(Fr)
    assert res < 1e-6 * (1 + 1e-6), res
    _, it64, _, _, _ = o.solve(F, tol=1e-6)
    assert st.iterations <= it64 + (3 if precision == "fp32" else 8)
    print(f"{name} {precision}: iters {st.iterations} (fp64 oracle {it64}), "
          f"rel. error vs FP64 oracle {_rel(Uh, U_ref):.2e}")


def test_nonhomogeneous_dirichlet_patch_test(built):
    p = meshgen.make_problem(None, dim=2, n=12, jitter=0.2, seed=11, E=5.0, nu=0.4)
    X = p["coords"]
    u = 0.3 + X @ np.array([[0.2, -0.5], [0.7, 0.1]]).T
    bnd = np.nonzero(np.any((X == 0.0) | (X == 1.0), axis=1))[0]
    dofs = (bnd[:, None] * 2 + np.arange(2)).ravel().astype(np.int64)
    p["dirichlet_dofs"] = dofs
    p["dirichlet_values"] = u.ravel()[dofs]
    s = vasmg.Solver(p, stream=torch.cuda.current_stream().cuda_stream)
    o = oracle.Oracle(p)
    np.testing.assert_allclose(s.export(vasmg.EXPORT_LIFT, 0, np.float64), o.export(oracle.LIFT, 0, np.float64),
                               rtol=1e-12, atol=1e-14)
    F = torch.zeros(X.shape[0] * 2, dtype=torch.float64, device="cuda")
    U = torch.zeros_like(F)
    rc, st, _ = s.solve(F, U, tol=1e-12)
    assert rc == 0
    np.testing.assert_allclose(U.cpu().numpy(), u.ravel(), atol=1e-9)
    s.close()


def test_edge_cases(built):
    stream = torch.cuda.current_stream().cuda_stream
    # zero right-hand side: no iterations, U = 0
    p = _prob("2d_n24")
    s = vasmg.Solver(p, stream=stream)
    F = torch.zeros(p["coords"].shape[0] * 2, dtype=torch.float64, device="cuda")
    U = torch.ones_like(F)
    rc, st, _ = s.solve(F, U)
    assert rc == 0 and st.iterations == 0 and float(U.abs().max()) == 0.0
    # host (numpy) vectors work as well
    o = oracle.Oracle(p)
    Fh = o.assemble_load(p["body_force"])
    Uh = np.zeros_like(Fh)
    rc, st, _ = s.solve(Fh, Uh, tol=1e-6)
    U_ref, it_ref, _, _, _ = o.solve(Fh, tol=1e-6)
    assert rc == 0 and _rel(Uh, U_ref) <= 1e-10
    # max_iters reached -> NOT_CONVERGED with the last iterate
    s2 = vasmg.Solver(p, stream=stream, max_iters=2)
    U2 = np.zeros_like(Fh)
    rc, st, _ = s2.solve(Fh, U2, tol=1e-12)
    assert rc == vasmg.VASMG_NOT_CONVERGED and st.iterations == 2
    # host loop instead of the conditional graph gives the same iterates, bit for bit
    s3 = vasmg.Solver(p, stream=stream, use_graph=False)
    U3 = np.zeros_like(Fh)
    rc, st3, _ = s3.solve(Fh, U3, tol=1e-6)
    assert rc == 0 and st3.iterations == it_ref and np.array_equal(U3, Uh)
    # repeated solves are deterministic
    U4 = np.zeros_like(Fh)
    s.solve(Fh, U4, tol=1e-6)
    assert np.array_equal(U4, Uh)
    # a 2x2-vertex mesh: the root is the only leaf (N <= T)
    tiny = meshgen.make_problem(None, dim=2, n=2, jitter=0.0, seed=1)
    tiny["dirichlet_dofs"] = np.array([0, 1, 3], dtype=np.int64)
    st_ = vasmg.Solver(tiny, stream=stream)
    ot = oracle.Oracle(tiny)
    assert st_.num_levels == ot.num_levels
    Ft = ot.assemble_load(tiny["body_force"])
    Ut = np.zeros_like(Ft)
    rc, _, _ = st_.solve(Ft, Ut, tol=1e-10)
    Ur, _, _, _, _ = ot.solve(Ft, tol=1e-10)
    assert rc == 0 and _rel(Ut, Ur) < 1e-10
    # single level (direct solve) with coarse_max_dofs
    small = meshgen.make_problem(None, dim=2, n=6, seed=2)
    ss = vasmg.Solver(small, stream=stream, coarse_max_dofs=200)
    os_ = oracle.Oracle(small, coarse_max_dofs=200)
    assert ss.num_levels == 1 == os_.num_levels
    Fs = os_.assemble_load(small["body_force"])
    Us = np.zeros_like(Fs)
    rc, sts, _ = ss.solve(Fs, Us, tol=1e-10)
    Ur, itr, _, _, _ = os_.solve(Fs, tol=1e-10)
    assert rc == 0 and _rel(Us, Ur) < 1e-10 and sts.iterations == itr
    # degenerate element is rejected
    bad = meshgen.make_problem(None, dim=2, n=4, seed=2)
    bad["elems"] = bad["elems"].copy()
    bad["elems"][0, 2] = bad["elems"][0, 1]
    with pytest.raises(vasmg.VasmgError) as ei:
        vasmg.Solver(bad, stream=stream)
    assert ei.value.code == vasmg.VASMG_ERR_DEGENERATE_ELEMENT
    # out-of-range element id is rejected
    bad2 = meshgen.make_problem(None, dim=2, n=4, seed=2)
    bad2["elems"] = bad2["elems"].copy()
    bad2["elems"][0, 0] = 10 ** 6
    with pytest.raises(vasmg.VasmgError) as ei:
        vasmg.Solver(bad2, stream=stream)
    assert ei.value.code == vasmg.VASMG_ERR_INVALID_ARG


@pytest.mark.parametrize("dim,k", [(2, 4), (3, 3)])
def test_theorem_3_2_on_device(built, dim, k):
    """Leaf capacity 9 (27) on a uniform grid: the device builds exactly the
    oracle's textbook-GMG hierarchy."""
    p = meshgen.make_problem(None, dim=dim, n=2 ** k + 1, jitter=0.0, seed=1)
    T = 9 if dim == 2 else 27
    o = oracle.Oracle(p, threshold=T)
    s = vasmg.Solver(p, stream=torch.cuda.current_stream().cuda_stream, threshold=T)
    assert s.num_levels == o.num_levels == k + 1
    for l in range(o.num_levels - 1):
        assert np.array_equal(s.export(vasmg.EXPORT_P_W, l, np.float64), o.prolongation(l)[2])
        assert np.array_equal(s.export(vasmg.EXPORT_P_CI, l, np.int32), o.prolongation(l)[1])


@pytest.mark.parametrize("T", [4, 8, 9])
@pytest.mark.parametrize("dim,n", [(2, 40), (3, 9)])
def test_threshold_sweep_matches_oracle(built, dim, n, T):
    """Leaf threshold T in {4, 8, 9} (the paper's 4 and two coarser trees):
    the same hierarchy as the oracle, bit for bit, and the same FP64 solve."""
    p = meshgen.make_problem(None, dim=dim, n=n, jitter=0.2 if dim == 2 else 0.15, seed=60 + n, nu=0.35)
    o = oracle.Oracle(p, threshold=T)
    s = vasmg.Solver(p, stream=torch.cuda.current_stream().cuda_stream, threshold=T)
    try:
        assert s.num_levels == o.num_levels
        for l in range(o.num_levels - 1):
            orp, oci, ow = o.prolongation(l)
            assert np.array_equal(s.export(vasmg.EXPORT_P_RP, l, np.int64), orp)
            assert np.array_equal(s.export(vasmg.EXPORT_P_CI, l, np.int32), oci)
            assert np.array_equal(s.export(vasmg.EXPORT_P_W, l, np.float64), ow)
        for l in range(o.num_levels):
            assert np.array_equal(s.export(vasmg.EXPORT_A_CI, l, np.int32), o.operator(l)[1])
            assert np.array_equal(s.export(vasmg.EXPORT_COLOUR, l, np.int32), o.colours(l))
        F = o.assemble_load(p["body_force"])
        U_ref, it_ref, _, _, _ = o.solve(F, tol=1e-6)
        U = np.zeros_like(F)
        rc, st, _ = s.solve(F, U, tol=1e-6)
        assert rc == 0 and abs(st.iterations - it_ref) <= 1 and _rel(U, U_ref) <= 1e-10
    finally:
        s.close()


@pytest.mark.parametrize("seed", range(6))
def test_random_problems(built, seed):
    p = meshgen.random_problem(seed)
    o = oracle.Oracle(p)
    s = vasmg.Solver(p, stream=torch.cuda.current_stream().cuda_stream)
    assert s.num_levels == o.num_levels
    for l in range(o.num_levels):
        assert np.array_equal(s.export(vasmg.EXPORT_COLOUR, l, np.int32), o.colours(l))
    F = o.assemble_load(p["body_force"])
    U_ref, it_ref, _, _, _ = o.solve(F, tol=1e-6)
    U = np.zeros_like(F)
    rc, st, _ = s.solve(F, U, tol=1e-6)
    assert rc == 0 and abs(st.iterations - it_ref) <= 1 and _rel(U, U_ref) <= 1e-10
