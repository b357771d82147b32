"""vasmg_solve_batch with one launch per level and phase across meshes.

Uneven 2D and 3D meshes (some with region levels, some small enough to run
entirely in the cluster tail) set up with one FP32-vector precision are solved
together: each region level's sweeps, residuals and transfers of all of them
in one launch, their tails in one launch, every CG kernel in one launch.
Checked:
  - every solution, iteration count and residual history is bitwise the one
    vasmg_solve gives for that mesh alone (FP32 and BF16 operator values);
  - the batch's launches do not grow with the number of meshes: at most
    3 + (5 R + 6) per iteration, R the most region levels of any mesh, and
    fewer than the single solves' launches together;
  - handles that cannot share launches (another precision among them, or one
    handle twice) still give the single solves' results.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2505_09064_gb300 import meshgen, vasmg  # noqa: E402

pytestmark = pytest.mark.gpu

MESHES = [
    dict(dim=2, n=24, jitter=0.2, seed=51),
    dict(dim=3, n=9, jitter=0.15, seed=52, nu=0.4),
    dict(dim=2, n=181, jitter=0.2, seed=53, checker=True),
    dict(dim=3, n=33, jitter=0.15, seed=54),
    dict(dim=3, n=17, jitter=0.0, seed=55, nu=0.45, graded=16.0),
    dict(dim=2, n=97, jitter=0.2, seed=56, E=30.0, nu=0.25),
]


@pytest.fixture(scope="module")
def built():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)
    return True


def _loads(solvers, probs, seed):
    rs = meshgen.Stream(seed)
    out = []
    for s, p in zip(solvers, probs):
        F = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        s.assemble_load(rs.uniform(p["dim"], -1.0, 1.0), F)
        out.append(F)
    return out


def _region_levels(s):
    return int(np.count_nonzero(s.export(vasmg.EXPORT_LANES, 0, np.int32)))


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_batch_one_launch_per_level_equals_single(built, precision):
    probs = [meshgen.make_problem(None, **m) for m in MESHES]
    stream = torch.cuda.current_stream().cuda_stream
    solvers = [vasmg.Solver(p, precision=precision, stream=stream, max_ctas=40) for p in probs]
    try:
        Fs = _loads(solvers, probs, 5)
        Us = [torch.full_like(F, float("nan")) for F in Fs]
        rc, sts = vasmg.vasmg_solve_batch([s.h for s in solvers], Fs, Us, tol=1e-6)
        assert rc == 0
        batch_launches = vasmg.vasmg_last_launch_count(solvers[0].h)
        single_launches = 0
        its = []
        for i, s in enumerate(solvers):
            U1 = torch.zeros_like(Fs[i])
            rc1, st1, _ = s.solve(Fs[i], U1, tol=1e-6)
            assert rc1 == 0
            single_launches += vasmg.vasmg_last_launch_count(s.h)
            assert sts[i].iterations == st1.iterations, (i, sts[i].iterations, st1.iterations)
            assert torch.equal(Us[i], U1), (i, float((Us[i] - U1).abs().max()))
            its.append(st1.iterations)
        R = max(_region_levels(s) for s in solvers)
        assert R >= 2
        assert batch_launches <= 3 + (5 * R + 6) * (max(its) + 1), (batch_launches, R, its)
        assert batch_launches < single_launches
        print(f"\n{precision}: {len(solvers)} meshes, iterations {its}, batch launches {batch_launches} "
              f"against {single_launches} for the single solves")
    finally:
        for s in solvers:
            s.close()


def test_batch_residual_history_equals_single(built):
    probs = [meshgen.make_problem(None, **m) for m in MESHES[:3]]
    stream = torch.cuda.current_stream().cuda_stream
    solvers = [vasmg.Solver(p, precision="fp32", stream=stream, max_ctas=64) for p in probs]
    try:
        Fs = _loads(solvers, probs, 6)
        Us = [torch.zeros_like(F) for F in Fs]
        lib = vasmg.load()
        import ctypes as C
        k = len(solvers)
        H = (C.c_void_p * k)(*[s.h.value for s in solvers])
        Fp = (C.c_void_p * k)(*[F.data_ptr() for F in Fs])
        Up = (C.c_void_p * k)(*[U.data_ptr() for U in Us])
        st = (vasmg.vasmg_stats * k)()
        hists = [np.zeros(300) for _ in range(k)]
        for i in range(k):
            st[i].res_history = hists[i].ctypes.data_as(C.c_void_p)
            st[i].res_history_cap = 300
        assert lib.vasmg_solve_batch(k, H, Fp, Up, 1e-6, st) == 0
        for i, s in enumerate(solvers):
            U1 = torch.zeros_like(Fs[i])
            rc1, st1, h1 = s.solve(Fs[i], U1, tol=1e-6, history_cap=300)
            assert np.array_equal(hists[i][: st1.iterations], h1)
    finally:
        for s in solvers:
            s.close()


def test_batch_falls_back_when_launches_cannot_be_shared(built):
    probs = [meshgen.make_problem(None, **m) for m in MESHES[:3]]
    stream = torch.cuda.current_stream().cuda_stream
    solvers = [vasmg.Solver(probs[0], precision="fp32", stream=stream, max_ctas=64),
               vasmg.Solver(probs[1], precision="fp64", stream=stream, max_ctas=64),
               vasmg.Solver(probs[2], precision="fp32", stream=stream, max_ctas=64)]
    try:
        Fs = _loads(solvers, probs, 7)
        # mixed precisions, and the same handle twice
        for hs, fs in (([s.h for s in solvers], Fs), ([solvers[0].h, solvers[0].h], [Fs[0], Fs[0]])):
            Us = [torch.zeros_like(F) for F in fs]
            rc, sts = vasmg.vasmg_solve_batch(hs, fs, Us, tol=1e-6)
            assert rc == 0
            for h, F, U in zip(hs, fs, Us):
                s = next(x for x in solvers if x.h.value == h.value)
                U1 = torch.zeros_like(F)
                s.solve(F, U1, tol=1e-6)
                assert torch.equal(U, U1)
    finally:
        for s in solvers:
            s.close()
