"""Lanes per row chosen by measurement (vasmg_options.autotune).

* Every region level (above the tail launch) gets one of 4, 8, 16, 32 lanes;
  the levels the tail runs report 0.
* The choice is kept per level signature for the process: a second handle of
  the same problem (here with a capped sweep grid) sweeps with the same lanes
  and returns the same bits.
* With autotune = 0 the lanes follow the rule from the mean number of
  off-diagonal blocks per row.
* The FP64 solve with the measured lanes equals the one with the rule's lanes
  to 1e-10 (the lane count changes only the order of additions in a row).
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2505_09064_gb300 import meshgen, vasmg  # noqa: E402

pytestmark = pytest.mark.gpu

CASES = {
    "2d_n300": dict(dim=2, n=300, jitter=0.2, seed=71, checker=True, E=100.0),
    "3d_n40": dict(dim=3, n=40, jitter=0.15, seed=72, nu=0.35),
}


@pytest.fixture(scope="module")
def built():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)
    return True


def _rule(avg):
    return 4 if avg <= 6.0 else 8 if avg <= 48.0 else 16 if avg <= 64.0 else 32


def _solve(s, prob):
    F = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    s.assemble_load(prob["body_force"], F)
    U = torch.zeros_like(F)
    rc, st, _ = s.solve(F, U, 1e-6)
    assert rc == 0 and st.rel_res < 1e-6
    return U.cpu().numpy(), st.iterations


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_autotuned_lanes(built, name, precision):
    prob = meshgen.make_problem(None, **CASES[name])
    st = torch.cuda.current_stream().cuda_stream
    a = vasmg.Solver(prob, precision=precision, stream=st)
    b = vasmg.Solver(prob, precision=precision, stream=st, max_ctas=64)
    r = vasmg.Solver(prob, precision=precision, stream=st, autotune=False)
    try:
        ga = a.export(vasmg.EXPORT_LANES, 0, np.int32)
        assert ga.size == a.num_levels
        region = ga > 0
        assert region[0] and set(ga[region].tolist()) <= {4, 8, 16, 32}
        # region levels first, then the tail's levels
        k = int(region.sum())
        assert region[:k].all() and not region[k:].any()
        assert np.array_equal(b.export(vasmg.EXPORT_LANES, 0, np.int32), ga)
        gr = r.export(vasmg.EXPORT_LANES, 0, np.int32)
        for l in range(k):
            nv, nnzb, _ = r.level_info(l)
            assert gr[l] == _rule((nnzb - nv) / nv)  # off-diagonal blocks per row
        Ua, ita = _solve(a, prob)
        Ub, itb = _solve(b, prob)
        assert ita == itb and np.array_equal(Ua, Ub)
        Ur, itr = _solve(r, prob)
        assert abs(ita - itr) <= 1
        if precision == "fp64":
            assert np.max(np.abs(Ua - Ur)) <= 1e-10 * np.max(np.abs(Ur))
        else:
            assert np.max(np.abs(Ua - Ur)) <= 1e-5 * np.max(np.abs(Ur))
    finally:
        for s in (a, b, r):
            s.close()
