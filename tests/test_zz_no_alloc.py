"""vasmg_coarse_solve_noalloc against vasmg_apply(VASMG_OP_COARSE).

The no-alloc entry point runs the same FP64 substitution with static device
scratch instead of per-call buffers; both must give the same solution (to
1e-13 relative, same arithmetic order), on two calls in a row.  The file is
named to be collected last, and each case also holds when run alone.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2505_09064_gb300 import meshgen, vasmg  # noqa: E402

pytestmark = pytest.mark.gpu

CASES = {
    # coarsened to the root cell: 2^d vertices on the coarsest level
    "2d_root": (dict(dim=2, n=24, jitter=0.2, seed=11), 0),
    # stopped early: a larger dense coarsest level (up to 4096 dofs)
    "2d_coarse_900": (dict(dim=2, n=40, jitter=0.2, seed=12), 900),
    "3d_coarse_600": (dict(dim=3, n=9, jitter=0.15, seed=13), 600),
}


@pytest.fixture(scope="module")
def built():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)
    return True


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("name", sorted(CASES))
def test_noalloc_coarse_solve_matches_apply(built, name):
    kw, cmax = CASES[name]
    prob = meshgen.make_problem(None, **kw)
    stream = torch.cuda.current_stream().cuda_stream
    s = vasmg.Solver(prob, precision="fp64", stream=stream, coarse_max_dofs=cmax)
    try:
        L = s.num_levels
        n = s.level_info(L - 1)[0] * s.dim
        assert 0 < n <= 4096
        rs = meshgen.Stream(500 + n)
        b = torch.tensor(rs.uniform(n, -1.0, 1.0), dtype=torch.float64, device="cuda")
        ref = torch.zeros(n, dtype=torch.float64, device="cuda")
        s.apply(vasmg.OP_COARSE, L - 1, b, ref)
        ref_h = ref.cpu().numpy()
        outs = []
        for _ in range(2):
            x = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
            vasmg.vasmg_coarse_solve_noalloc(s.h, b, x, stream)
            torch.cuda.synchronize()
            outs.append(x.cpu().numpy())
        for x in outs:
            assert np.all(np.isfinite(x))
            assert _rel(x, ref_h) <= 1e-13
        assert np.array_equal(outs[0], outs[1])
        # in place (b and x the same buffer)
        y = b.clone()
        vasmg.vasmg_coarse_solve_noalloc(s.h, y, y, stream)
        torch.cuda.synchronize()
        assert _rel(y.cpu().numpy(), ref_h) <= 1e-13
    finally:
        s.close()
