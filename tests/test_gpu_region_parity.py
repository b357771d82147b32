"""Whole FP64 solves against the oracle at sizes that run the region launches.

Levels with more than 20,000 vertices are smoothed by the cooperative region
kernels (forward sweep, residual, restriction, prolongation, backward sweep),
the smaller ones by the cluster tail kernel; the FP64 outer CG uses the SELL
SpMV.  Every case here has at least two region levels, so the whole path the
benchmark runs (region levels -> tail -> coarsest Cholesky -> back up, inside
PCG) is compared with the oracle (Alg. 2 with Alg. 3 as the preconditioner,
stop rule of Sec. 5):

  - FP64: solution element by element (max norm) to 1e-10 relative, the same
    iteration count +-1, and the residual history to 1e-8;
  - one V-cycle from level 0 against the oracle's, element by element, 1e-11;
  - FP32 V-cycle and BF16 operator values: the true residual of the returned
    solution below 1e-6 (the tolerance), its error against the FP64 oracle
    solution printed.

Inputs: the unit-square and unit-cube recipes at 257^2, 321^2, 33^3 and 41^3
vertices, a 1:100 checkerboard of Young's moduli, and the paper's four 2D
geometries (Sec. 5) at 30-45 % of the paper's vertex counts.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2505_09064_gb300 import meshgen, vasmg  # noqa: E402

pytestmark = pytest.mark.gpu

TAIL_NV = 20000
TOL = 1e-6

CASES = {
    "2d_257": ("grid", dict(dim=2, n=257, jitter=0.2, seed=21)),
    "2d_257_checker": ("grid", dict(dim=2, n=257, jitter=0.2, seed=22, checker=True)),
    "2d_321_nu045": ("grid", dict(dim=2, n=321, jitter=0.2, seed=25, nu=0.45)),
    "3d_33": ("grid", dict(dim=3, n=33, jitter=0.15, seed=23)),
    "3d_41": ("grid", dict(dim=3, n=41, jitter=0.15, seed=24)),
    "hole_round": ("paper", 0.45),
    "ring": ("paper", 0.3),
    "hole_square": ("paper", 0.3),
    "dam": ("paper", 0.3),
}


@pytest.fixture(scope="module")
def built():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)
    return True


_cache = {}


def case(name):
    if name not in _cache:
        kind, arg = CASES[name]
        if kind == "grid":
            p = meshgen.make_problem(None, **arg)
        else:
            p = meshgen.paper_example(name, arg)
        o = oracle.Oracle(p)
        F = p["F"] if "F" in p else o.assemble_load(p["body_force"])
        U_ref, it_ref, _, st_ref, hist_ref = o.solve(F, tol=TOL, hist_cap=500)
        assert st_ref == 0
        _cache.clear()  # one case's oracle at a time
        _cache[name] = (p, o, F, U_ref, it_ref, hist_ref)
    return _cache[name]


def _maxrel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _region_levels(s):
    lanes = s.export(vasmg.EXPORT_LANES, 0, np.int32)
    return int(np.count_nonzero(lanes))


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_region_solve_matches_oracle(built, name):
    p, o, F, U_ref, it_ref, hist_ref = case(name)
    s = vasmg.Solver(p, precision="fp64", stream=torch.cuda.current_stream().cuda_stream)
    try:
        assert s.num_levels == o.num_levels
        nv = [s.level_info(l)[0] for l in range(s.num_levels)]
        assert sum(1 for v in nv[:-1] if v > TAIL_NV) >= 2, nv
        assert _region_levels(s) >= 2
        Fd = torch.from_numpy(F).cuda()
        U = torch.zeros_like(Fd)
        rc, st, hist = s.solve(Fd, U, tol=TOL, history_cap=500)
        assert rc == 0
        assert abs(st.iterations - it_ref) <= 1, (st.iterations, it_ref)
        err = _maxrel(U.cpu().numpy(), U_ref)
        assert err <= 1e-10, err
        k = min(len(hist), len(hist_ref))
        np.testing.assert_allclose(hist[:k], hist_ref[:k], rtol=1e-8)
        # one V-cycle from level 0: region levels, tail, coarsest solve, back up
        d = p["dim"]
        rs = meshgen.Stream(91)
        b = rs.uniform(nv[0] * d, -1.0, 1.0)
        b[o.dead(0).astype(bool)] = 0.0
        y = torch.zeros(b.size, dtype=torch.float64, device="cuda")
        s.apply(vasmg.OP_VCYCLE, 0, torch.from_numpy(b).cuda(), y)
        verr = _maxrel(y.cpu().numpy(), o.vcycle(b, level=0))
        assert verr <= 1e-11, verr
        print(f"{name}: levels {nv}, iterations {st.iterations} (oracle {it_ref}), "
              f"max-norm error {err:.2e}, V-cycle {verr:.2e}")
    finally:
        s.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("name", ["2d_257_checker", "3d_41", "hole_square"])
def test_mixed_precision_region_solve(built, name, precision):
    p, o, F, U_ref, it_ref, _ = case(name)
    s = vasmg.Solver(p, precision=precision, stream=torch.cuda.current_stream().cuda_stream)
    try:
        Fd = torch.from_numpy(F).cuda()
        U = torch.zeros_like(Fd)
        rc, st, _ = s.solve(Fd, U, tol=TOL)
        assert rc == 0 and st.rel_res < TOL
        Uh = U.cpu().numpy()
        Fr = F.copy()
        Fr[p["dirichlet_dofs"]] = 0.0
        res = np.linalg.norm(Fr - o.apply_A(0, Uh)) / np.linalg.norm(Fr)
        assert res < TOL * (1 + 1e-6), res
        assert st.iterations <= it_ref + (3 if precision == "fp32" else 10)
        print(f"{name} {precision}: iterations {st.iterations} (FP64 oracle {it_ref}), true residual {res:.2e}, "
              f"max-norm error vs FP64 oracle {_maxrel(Uh, U_ref):.2e}")
    finally:
        s.close()
