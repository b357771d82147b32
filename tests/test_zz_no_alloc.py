"""vasmg_coarse_solve_noalloc: the coarsest-level solve that allocates nothing.

Some callers cannot allocate device memory in the middle of a solve: a request
server that has budgeted every byte of device memory per request (an
allocation could exceed the budget or block on the allocator), or a tight
latency-bound loop that must never enter the allocator.  For them the library
offers this entry point, which keeps its scratch in a fixed static device
array instead of allocating per call.

Checked here, on two calls in a row and in place:
  - it equals vasmg_apply(VASMG_OP_COARSE) (the allocating path, same FP64
    substitution) to 1e-13 relative, max norm, on FP64 handles; on FP32 and
    BF16-smoother handles vasmg_apply stages its vectors in the V-cycle's
    FP32 precision while this entry point stays in FP64, so there the two
    agree to FP32 rounding (1e-5);
  - it equals the CPU oracle's coarsest solve (its own Cholesky factor) to
    1e-10 relative, max norm;
  - for FP64, FP32 and BF16-smoother handles (every mode keeps the FP64
    factor);
  - a host pointer handed straight to the C entry point is refused, and so is
    a vector of the wrong length.

The file is named to be collected last; each case also holds when run alone
in a fresh process.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
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


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_noalloc_coarse_solve_matches_apply_and_oracle(built, name, precision):
    kw, cmax = CASES[name]
    prob = meshgen.make_problem(None, **kw)
    stream = torch.cuda.current_stream().cuda_stream
    s = vasmg.Solver(prob, precision=precision, stream=stream, coarse_max_dofs=cmax)
    try:
        L = s.num_levels
        n = s.level_info(L - 1)[0] * s.dim
        assert 0 < n <= vasmg.NOALLOC_MAX_DOFS
        rs = meshgen.Stream(500 + n)
        b_h = rs.uniform(n, -1.0, 1.0)
        b = torch.tensor(b_h, dtype=torch.float64, device="cuda")
        ref = torch.zeros(n, dtype=torch.float64, device="cuda")
        s.apply(vasmg.OP_COARSE, L - 1, b, ref)
        ref_h = ref.cpu().numpy()
        o = oracle.Oracle(prob, coarse_max_dofs=cmax)
        assert o.num_levels == L
        x_or = o.coarse_solve(b_h)
        outs = []
        for _ in range(2):
            x = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
            s.coarse_solve_noalloc(b, x, stream)
            torch.cuda.synchronize()
            outs.append(x.cpu().numpy())
        tol_apply = 1e-13 if precision == "fp64" else 1e-5
        for x in outs:
            assert np.all(np.isfinite(x))
            assert _rel(x, ref_h) <= tol_apply
            assert _rel(x, x_or) <= 1e-10
        assert np.array_equal(outs[0], outs[1])
        # in place (b and x the same buffer)
        y = b.clone()
        s.coarse_solve_noalloc(y, y, stream)
        torch.cuda.synchronize()
        assert np.array_equal(y.cpu().numpy(), outs[0])
    finally:
        s.close()


def test_noalloc_refuses_bad_vectors(built):
    kw, cmax = CASES["2d_root"]
    prob = meshgen.make_problem(None, **kw)
    stream = torch.cuda.current_stream().cuda_stream
    s = vasmg.Solver(prob, stream=stream, coarse_max_dofs=cmax)
    try:
        n = s.level_info(s.num_levels - 1)[0] * s.dim
        lib = vasmg.load()
        # host memory handed straight to the C entry point is refused before any launch
        bh = np.ones(n)
        xh = np.zeros(n)
        rc = lib.vasmg_coarse_solve_noalloc(s.h, bh.ctypes.data_as(C.c_void_p), xh.ctypes.data_as(C.c_void_p),
                                            C.c_void_p(stream))
        assert rc == vasmg.VASMG_ERR_INVALID_ARG
        assert np.all(xh == 0.0)
        bd = torch.ones(n, dtype=torch.float64, device="cuda")
        rc = lib.vasmg_coarse_solve_noalloc(s.h, C.c_void_p(bd.data_ptr()), xh.ctypes.data_as(C.c_void_p),
                                            C.c_void_p(stream))
        assert rc == vasmg.VASMG_ERR_INVALID_ARG
        # the binding refuses a device vector of the wrong length
        with pytest.raises(ValueError):
            s.coarse_solve_noalloc(bd, torch.zeros(n + 1, dtype=torch.float64, device="cuda"), stream)
        # a good call still works afterwards
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        s.coarse_solve_noalloc(bd, x, stream)
        torch.cuda.synchronize()
        assert np.all(np.isfinite(x.cpu().numpy()))
    finally:
        s.close()
