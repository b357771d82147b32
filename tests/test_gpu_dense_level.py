"""The dense level of the FP32 V-cycle against the recursion it replaces.

With vasmg_options.dense_coarse = 1 (the default) the FP32-vector modes apply
the V-cycle from a small level k down to the coarsest as one precomputed
matrix M (the cycle applied to the unit vectors at setup).  It is the same
linear operator, so against the same handle built with dense_coarse = 0:

* the V-cycle from every level at or above k agrees to FP32 rounding, and
  below k, where the dense level is not used, bitwise;
* PCG takes the same number of iterations (within one) to a solution that
  agrees to the tolerance;
* after vasmg_update_data the matrix is rebuilt for the new values;
* the FP64 path has no dense level.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2505_09064_gb300 import meshgen, vasmg  # noqa: E402

pytestmark = pytest.mark.gpu

CASES = {
    # the whole hierarchy in the tail, one CTA
    "2d_n40": dict(dim=2, n=40, jitter=0.2, seed=81),
    # region levels above the tail, a cluster tail
    "2d_n300_checker": dict(dim=2, n=300, jitter=0.2, seed=82, checker=True, E=100.0),
    "3d_n12": dict(dim=3, n=12, jitter=0.15, seed=83, nu=0.4),
    "3d_n40": dict(dim=3, n=40, jitter=0.15, seed=84),
}


@pytest.fixture(scope="module")
def built():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)
    return True


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _pair(prob, precision="fp32"):
    st = torch.cuda.current_stream().cuda_stream
    return (vasmg.Solver(prob, precision=precision, stream=st, dense_coarse=True),
            vasmg.Solver(prob, precision=precision, stream=st, dense_coarse=False))


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_dense_level_is_the_same_operator(built, name, precision):
    prob = meshgen.make_problem(None, **CASES[name])
    d = prob["dim"]
    sd, sr = _pair(prob, precision)
    try:
        k, nk = (int(v) for v in sd.export(vasmg.EXPORT_DENSE, 0, np.int64))
        assert 0 <= k < sd.num_levels and nk == sd.level_info(k)[0] * d
        assert tuple(sr.export(vasmg.EXPORT_DENSE, 0, np.int64)) == (-1, 0)
        rs = meshgen.Stream(90)
        for l in range(sd.num_levels):
            nl = sd.level_info(l)[0] * d
            dead = sd.export(vasmg.EXPORT_DEAD, l, np.uint8).astype(bool)
            b = rs.uniform(nl, -1.0, 1.0)
            b[dead] = 0.0
            yd = torch.zeros(nl, dtype=torch.float64, device="cuda")
            yr = torch.zeros(nl, dtype=torch.float64, device="cuda")
            bd = torch.from_numpy(b).cuda()
            sd.apply(vasmg.OP_VCYCLE, l, bd, yd)
            sr.apply(vasmg.OP_VCYCLE, l, bd, yr)
            yd, yr = yd.cpu().numpy(), yr.cpu().numpy()
            if l > k:
                assert np.array_equal(yd, yr), l
            else:
                assert _rel(yd, yr) <= 1e-4, (l, _rel(yd, yr))
        F = torch.zeros(sd.n, dtype=torch.float64, device="cuda")
        sd.assemble_load(prob["body_force"], F)
        Ud, Ur = torch.zeros_like(F), torch.zeros_like(F)
        rc1, st1, _ = sd.solve(F, Ud, 1e-6)
        rc2, st2, _ = sr.solve(F, Ur, 1e-6)
        assert rc1 == rc2 == 0 and st1.rel_res < 1e-6 and st2.rel_res < 1e-6
        assert abs(st1.iterations - st2.iterations) <= 1
        assert _rel(Ud.cpu().numpy(), Ur.cpu().numpy()) <= 1e-5
    finally:
        sd.close()
        sr.close()


def test_dense_level_rebuilt_by_update(built):
    prob = meshgen.make_problem(None, **CASES["2d_n300_checker"])
    q = dict(prob)
    q["lam"] = np.asarray(prob["lam"]) * 3.0
    q["mu"] = np.asarray(prob["mu"]) * 0.5
    st = torch.cuda.current_stream().cuda_stream
    s = vasmg.Solver(prob, precision="fp32", stream=st)
    fresh = vasmg.Solver(q, precision="fp32", stream=st)
    try:
        s.update(q)
        k = int(s.export(vasmg.EXPORT_DENSE, 0, np.int64)[0])
        assert k >= 0
        nk = s.level_info(k)[0] * 2
        b = torch.from_numpy(meshgen.Stream(91).uniform(nk, -1.0, 1.0)).cuda()
        b[torch.from_numpy(s.export(vasmg.EXPORT_DEAD, k, np.uint8).astype(bool)).cuda()] = 0.0
        y1 = torch.zeros(nk, dtype=torch.float64, device="cuda")
        y2 = torch.zeros(nk, dtype=torch.float64, device="cuda")
        s.apply(vasmg.OP_VCYCLE, k, b, y1)
        fresh.apply(vasmg.OP_VCYCLE, k, b, y2)
        assert torch.equal(y1, y2)
    finally:
        s.close()
        fresh.close()


def test_fp64_has_no_dense_level(built):
    prob = meshgen.make_problem(None, **CASES["2d_n40"])
    s = vasmg.Solver(prob, precision="fp64", stream=torch.cuda.current_stream().cuda_stream)
    try:
        assert tuple(s.export(vasmg.EXPORT_DENSE, 0, np.int64)) == (-1, 0)
    finally:
        s.close()
