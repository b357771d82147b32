"""The paper's cycle variants on the GPU against the oracle's.

  - W-cycle (Fig. 2; vasmg_options.cycle = 2): every level above the
    second-coarsest solves its coarse problem by two cycles, the second on the
    updated coarse residual; the coarsest level is solved once.
  - Additive form of Sec. 4 (vasmg_options.additive = 1): B = S + P B_1 P^T,
    S one forward and one backward sweep from zero on the fine level, B_1 the
    cycle from level 1.

Checked in FP64, element by element (max norm): the preconditioner applied to
a random vector against the oracle's (Oracle.set_cycle, Oracle.precondition)
to 1e-11, the cycle from every level to 1e-11, and whole solves to 1e-10 with
the same iteration count +-1, on small meshes and on meshes whose fine levels
run the region launches.  FP32 solves with the variants reach the 1e-6 true
residual.  Iteration counts are printed beside the V-cycle's.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2505_09064_gb300 import meshgen, vasmg  # noqa: E402

pytestmark = pytest.mark.gpu

SMALL = {
    "2d_24": dict(dim=2, n=24, jitter=0.2, seed=41),
    "2d_40_checker": dict(dim=2, n=40, jitter=0.2, seed=42, checker=True),
    "3d_8": dict(dim=3, n=8, jitter=0.15, seed=43),
    "3d_11_graded": dict(dim=3, n=11, jitter=0.0, seed=44, nu=0.45, graded=16.0),
}
REGION = {
    "2d_257": dict(dim=2, n=257, jitter=0.2, seed=21),
    "3d_33": dict(dim=3, n=33, jitter=0.15, seed=23),
}
VARIANTS = [(2, False), (1, True), (2, True)]


@pytest.fixture(scope="module")
def built():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)
    return True


def _maxrel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _check(prob, gamma, additive, single_steps, label):
    stream = torch.cuda.current_stream().cuda_stream
    o = oracle.Oracle(prob)
    o.set_cycle(gamma, additive)
    s = vasmg.Solver(prob, precision="fp64", stream=stream, cycle=gamma, additive=additive)
    try:
        assert s.num_levels == o.num_levels
        d = prob["dim"]
        rs = meshgen.Stream(17)
        if single_steps:
            n0 = o.nv_level(0) * d
            b = rs.uniform(n0, -1.0, 1.0)
            b[o.dead(0).astype(bool)] = 0.0
            y = torch.zeros(n0, dtype=torch.float64, device="cuda")
            s.apply(vasmg.OP_PRECOND, 0, torch.from_numpy(b).cuda(), y)
            err = _maxrel(y.cpu().numpy(), o.precondition(b))
            assert err <= 1e-11, (label, "precond", err)
            for l in range(o.num_levels):
                nl = o.nv_level(l) * d
                bl = rs.uniform(nl, -1.0, 1.0)
                bl[o.dead(l).astype(bool)] = 0.0
                yl = torch.zeros(nl, dtype=torch.float64, device="cuda")
                s.apply(vasmg.OP_VCYCLE, l, torch.from_numpy(bl).cuda(), yl)
                err = _maxrel(yl.cpu().numpy(), o.vcycle(bl, level=l))
                assert err <= 1e-11, (label, "cycle from level", l, err)
        F = prob["F"] if "F" in prob else o.assemble_load(prob["body_force"])
        U_ref, it_ref, _, st_ref, _ = o.solve(F, tol=1e-6)
        assert st_ref == 0
        U = np.zeros_like(F)
        rc, st, _ = s.solve(F, U, tol=1e-6)
        assert rc == 0
        assert abs(st.iterations - it_ref) <= 1, (label, st.iterations, it_ref)
        err = _maxrel(U, U_ref)
        assert err <= 1e-10, (label, err)
        return st.iterations
    finally:
        s.close()


@pytest.mark.parametrize("name", list(SMALL))
def test_variants_match_oracle_small(built, name):
    prob = meshgen.make_problem(None, **SMALL[name])
    its = {}
    for gamma, additive in [(1, False)] + VARIANTS:
        its[(gamma, additive)] = _check(prob, gamma, additive, True, f"{name} gamma={gamma} additive={additive}")
    print(f"\n{name}: iterations V {its[(1, False)]}, W {its[(2, False)]}, additive(V) {its[(1, True)]}, "
          f"additive(W) {its[(2, True)]}")


@pytest.mark.parametrize("name", list(REGION))
def test_variants_match_oracle_region_levels(built, name):
    prob = meshgen.make_problem(None, **REGION[name])
    its = {}
    for gamma, additive in VARIANTS:
        its[(gamma, additive)] = _check(prob, gamma, additive, False, f"{name} gamma={gamma} additive={additive}")
    print(f"\n{name}: iterations W {its[(2, False)]}, additive(V) {its[(1, True)]}, additive(W) {its[(2, True)]}")


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("name", ["2d_40_checker", "3d_11_graded"])
def test_variants_mixed_precision_converge(built, name, precision):
    prob = meshgen.make_problem(None, **SMALL[name])
    o = oracle.Oracle(prob)
    F = o.assemble_load(prob["body_force"])
    Fr = F.copy()
    Fr[prob["dirichlet_dofs"]] = 0.0
    stream = torch.cuda.current_stream().cuda_stream
    for gamma, additive in VARIANTS:
        s = vasmg.Solver(prob, precision=precision, stream=stream, cycle=gamma, additive=additive)
        try:
            U = np.zeros_like(F)
            rc, st, _ = s.solve(F, U, tol=1e-6)
            assert rc == 0
            res = np.linalg.norm(Fr - o.apply_A(0, U)) / np.linalg.norm(Fr)
            assert res < 1e-6 * (1 + 1e-6), (gamma, additive, res)
        finally:
            s.close()
