"""The staged region sweeps of 3D levels (vstaged_kernel).

The forward and backward sweeps of a 3D level above the tail threshold
stream their operator part from a second copy, laid out in per-thread slot
streams (each colour step's rows dealt to the lane groups longest first) and
copied into shared memory ahead of the rows.  Checked:

  - VASMG_EXPORT_STAGED: every 3D region level has both copies, with at least
    one slot per block and few padding slots; 2D levels and the tail's levels
    have none;
  - the staged sweeps of every region level in isolation against the oracle's
    multicolour block Gauss-Seidel sweep (Alg. 1 in the multicolour order),
    element by element: the forward sweep from zero and the backward sweep
    from an arbitrary start, in FP64, FP32 and BF16 operator values;
  - after vasmg_update_data with new Lame parameters, a solve is bitwise the
    solve of a fresh handle set up on the new data: the staged copies are
    refilled with the new values.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2505_09064_gb300 import meshgen, vasmg  # noqa: E402

pytestmark = pytest.mark.gpu

MESH3 = dict(dim=3, n=41, jitter=0.15, seed=61)
MESH2 = dict(dim=2, n=257, jitter=0.2, seed=62)


@pytest.fixture(scope="module")
def built():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)
    return True


def _solver(prob, precision):
    return vasmg.Solver(prob, precision=precision, stream=torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16"])
def test_staged_copies_per_level(built, precision):
    s3 = _solver(meshgen.make_problem(None, **MESH3), precision)
    s2 = _solver(meshgen.make_problem(None, **MESH2), precision)
    try:
        lanes = s3.export(vasmg.EXPORT_LANES, 0, np.int32)
        assert np.count_nonzero(lanes) >= 1
        for l in range(s3.num_levels):
            v = s3.export(vasmg.EXPORT_STAGED, l, np.int64)
            if lanes[l] == 0:
                assert not v.any(), (l, v)
                continue
            fwd_slots, lo_blocks, bwd_slots, blocks, slot_bytes = (int(a) for a in v)
            assert slot_bytes == 4 + 9 * {"fp64": 8, "fp32": 4, "bf16": 2}[precision]
            assert bwd_slots >= blocks > 0 and fwd_slots >= lo_blocks > 0
            # padding: rows rounded up to whole lane steps, streams to whole chunks
            assert bwd_slots <= 2.0 * blocks, (l, bwd_slots, blocks, int(lanes[l]))
            print(f"\n{precision} level {l}: G={int(lanes[l])} backward slots / blocks = {bwd_slots / blocks:.3f}, "
                  f"forward {fwd_slots / lo_blocks:.3f}")
        for l in range(s2.num_levels):
            assert not s2.export(vasmg.EXPORT_STAGED, l, np.int64).any()
    finally:
        s3.close()
        s2.close()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5), ("bf16", 2e-2)])
def test_staged_sweeps_against_oracle(built, precision, tol):
    p = meshgen.make_problem(None, **MESH3)
    o = oracle.Oracle(p)
    s = _solver(p, precision)
    try:
        lanes = s.export(vasmg.EXPORT_LANES, 0, np.int32)
        rs = meshgen.Stream(63)
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        checked = 0
        for l in range(s.num_levels - 1):
            if lanes[l] == 0:
                continue
            assert s.export(vasmg.EXPORT_STAGED, l, np.int64)[0] > 0
            nl = o.nv_level(l) * 3
            dead = o.dead(l).astype(bool)
            b = rs.uniform(nl, -1, 1)
            b[dead] = 0.0
            y = torch.zeros(nl, dtype=torch.float64, device="cuda")
            s.apply(vasmg.OP_SMOOTH_FWD, l, dev(b), y)
            assert _rel(y.cpu().numpy(), o.gs_sweep(l, b, np.zeros(nl), forward=True)) <= tol
            x0 = rs.uniform(nl, -1, 1)
            x0[dead] = 0.0
            y = dev(x0.copy())
            s.apply(vasmg.OP_SMOOTH_BWD, l, dev(b), y)
            assert _rel(y.cpu().numpy(), o.gs_sweep(l, b, x0, forward=False)) <= tol
            checked += 1
        assert checked >= 1
    finally:
        s.close()


@pytest.mark.parametrize("precision", ["fp64", "bf16"])
def test_update_refills_staged_copies(built, precision):
    p_old = meshgen.make_problem(None, **MESH3, nu=0.3)
    p_new = meshgen.make_problem(None, **MESH3, nu=0.45, E=7.0)
    a = _solver(p_old, precision)
    b = _solver(p_new, precision)
    try:
        F = torch.zeros(a.n, dtype=torch.float64, device="cuda")
        a.assemble_load(np.array([0.3, -1.0, 0.5]), F)
        U = torch.zeros_like(F)
        a.solve(F, U, tol=1e-6)
        a.update(p_new)
        Ua, Ub = torch.zeros_like(F), torch.zeros_like(F)
        rca, sta, _ = a.solve(F, Ua, tol=1e-6)
        rcb, stb, _ = b.solve(F, Ub, tol=1e-6)
        assert rca == 0 and rcb == 0
        assert sta.iterations == stb.iterations
        assert torch.equal(Ua, Ub), float((Ua - Ub).abs().max())
    finally:
        a.close()
        b.close()
