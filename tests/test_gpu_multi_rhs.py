"""vasmg_solve_multi: k right-hand sides on one hierarchy.

Every kernel of an iteration reads the operators once for all of them, but
each right-hand side follows exactly the arithmetic of a single vasmg_solve
(the same lanes per row, order of additions and reduction trees).  So for
every right-hand side the solution, the iteration count and the residual
history must be bitwise those of vasmg_solve alone -- for k = 2, 3, 5, 8 and
11 (passes of 2, 4 and 8 with padding, and more than one pass), in the FP32
and BF16-operator modes, on meshes whose levels run in the region launches
and on small ones that run entirely in the cluster tail, and with a zero
right-hand side among them.  The solutions are also checked against the FP64
oracle through the true residual.  FP64 handles run the k solves one after
another and must agree as well.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2505_09064_gb300 import meshgen, vasmg  # noqa: E402

pytestmark = pytest.mark.gpu

CASES = {
    "2d_24": dict(dim=2, n=24, jitter=0.2, seed=31),
    "3d_9": dict(dim=3, n=9, jitter=0.15, seed=32),
    "2d_257_checker": dict(dim=2, n=257, jitter=0.2, seed=33, checker=True),
    "3d_33": dict(dim=3, n=33, jitter=0.15, seed=34, nu=0.4),
    "3d_33_graded": dict(dim=3, n=33, jitter=0.0, seed=35, nu=0.45, graded=16.0),
}


@pytest.fixture(scope="module")
def built():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)
    return True


def _loads(s, prob, k, seed):
    """k right-hand sides: body-force loads with random directions, every
    third one a random vector (zero at Dirichlet dofs is not required)."""
    rs = meshgen.Stream(seed)
    d = prob["dim"]
    out = []
    for i in range(k):
        F = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        if i % 3 == 2:
            F.copy_(torch.from_numpy(rs.uniform(s.n, -1.0, 1.0)))
        else:
            s.assemble_load(rs.uniform(d, -1.0, 1.0), F)
        out.append(F)
    return out


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("name", list(CASES))
def test_multi_equals_single_bitwise(built, name, precision):
    prob = meshgen.make_problem(None, **CASES[name])
    stream = torch.cuda.current_stream().cuda_stream
    s = vasmg.Solver(prob, precision=precision, stream=stream)
    try:
        for k in (2, 3, 5, 8, 11):
            Fs = _loads(s, prob, k, 100 + k)
            Us = [torch.full_like(F, float("nan")) for F in Fs]
            rc, sts, hists = s.solve_multi(Fs, Us, tol=1e-6, history_cap=300)
            assert rc == 0
            for i in range(k):
                U1 = torch.zeros_like(Fs[i])
                rc1, st1, h1 = s.solve(Fs[i], U1, tol=1e-6, history_cap=300)
                assert rc1 == 0
                assert sts[i].iterations == st1.iterations, (k, i, sts[i].iterations, st1.iterations)
                assert torch.equal(Us[i], U1), (k, i, float((Us[i] - U1).abs().max()))
                assert np.array_equal(hists[i], h1)
                assert sts[i].rel_res == st1.rel_res
            if k == 8 and name in ("3d_33", "2d_257_checker"):
                print(f"{name} {precision} k=8: launches {vasmg.vasmg_last_launch_count(s.h)}, "
                      f"iterations {[st.iterations for st in sts]}")
    finally:
        s.close()


@pytest.mark.parametrize("name", ["2d_24", "3d_33"])
def test_multi_zero_rhs_and_oracle_residual(built, name):
    prob = meshgen.make_problem(None, **CASES[name])
    stream = torch.cuda.current_stream().cuda_stream
    s = vasmg.Solver(prob, precision="fp32", stream=stream)
    o = oracle.Oracle(prob)
    try:
        Fs = _loads(s, prob, 4, 7)
        Fs[1].zero_()
        Us = [torch.full_like(F, float("nan")) for F in Fs]
        rc, sts, _ = s.solve_multi(Fs, Us, tol=1e-6)
        assert rc == 0
        assert sts[1].iterations == 0 and float(Us[1].abs().max()) == 0.0
        dd = prob["dirichlet_dofs"]
        for i in (0, 2, 3):
            F = Fs[i].cpu().numpy().copy()
            F[dd] = 0.0
            U = Us[i].cpu().numpy()
            res = np.linalg.norm(F - o.apply_A(0, U)) / np.linalg.norm(F)
            assert res < 1e-6 * (1 + 1e-6), (i, res)
    finally:
        s.close()


def test_multi_fp64_handle_runs_single_solves(built):
    prob = meshgen.make_problem(None, **CASES["2d_24"])
    stream = torch.cuda.current_stream().cuda_stream
    s = vasmg.Solver(prob, precision="fp64", stream=stream)
    try:
        Fs = _loads(s, prob, 3, 9)
        Us = [torch.zeros_like(F) for F in Fs]
        rc, sts, _ = s.solve_multi(Fs, Us)
        assert rc == 0
        for i in range(3):
            U1 = torch.zeros_like(Fs[i])
            s.solve(Fs[i], U1)
            assert torch.equal(Us[i], U1)
    finally:
        s.close()


def test_multi_kernel_timing_hook(built):
    """The per-kernel timing of the multi launches reports the operator bytes
    once and the vectors once per right-hand side."""
    prob = meshgen.make_problem(None, **CASES["3d_33"])
    s = vasmg.Solver(prob, precision="fp32", stream=torch.cuda.current_stream().cuda_stream)
    try:
        ms1, b1 = vasmg.vasmg_time_kernel(s.h, vasmg.KERNEL_SWEEP, 1, 3)
        for k in (2, 4, 8):
            ms, b = vasmg.vasmg_time_kernel_multi(s.h, vasmg.KERNEL_SWEEP, 1, k, 3)
            assert ms > 0 and b > b1
        with pytest.raises(vasmg.VasmgError):
            vasmg.vasmg_time_kernel_multi(s.h, vasmg.KERNEL_SWEEP, 1, 3, 3)
    finally:
        s.close()
