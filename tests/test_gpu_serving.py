"""Batched and served solves: each result equals the same solve run alone.

The region decomposition of a sweep only changes which CTA computes a row,
not the arithmetic of any row, so a solve with capped sweep grids
(vasmg_options.max_ctas), run concurrently with others, must reproduce the
solve run alone: same iteration count, same U (to 1e-12 relative).
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2505_09064_gb300 import meshgen, vasmg  # noqa: E402

pytestmark = pytest.mark.gpu

MIX = [
    dict(dim=2, n=40, jitter=0.2, seed=21),
    dict(dim=3, n=10, jitter=0.15, seed=22, nu=0.4),
    dict(dim=2, n=73, jitter=0.2, seed=23, E=50.0, checker=True),
    dict(dim=3, n=13, jitter=0.0, seed=24, nu=0.45, graded=16.0),
    dict(dim=2, n=128, jitter=0.2, seed=25, nu=0.2),
]


@pytest.fixture(scope="module")
def built():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)
    return True


def _rhs(prob, k, seed):
    """k right-hand sides: the assembled body-force load, then random loads."""
    n = prob["coords"].shape[0] * prob["dim"]
    rs = meshgen.Stream(seed)
    out = []
    for i in range(k):
        F = rs.uniform(n, -1.0, 1.0)
        F[prob["dirichlet_dofs"]] = 0.0
        out.append(F)
    return out


def _alone(prob, Fs, precision, autotune=True):
    s = vasmg.Solver(prob, precision=precision, autotune=autotune)
    try:
        res = []
        for F in Fs:
            U = np.zeros_like(F)
            rc, st, _ = s.solve(F, U, 1e-6)
            assert rc == 0
            res.append((U, st.iterations))
        return res
    finally:
        s.close()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_solve_batch_concurrent_equals_alone(built, precision):
    probs = [meshgen.make_problem(None, **kw) for kw in MIX[:4]]
    Fs = [_rhs(p, 1, 100 + i)[0] for i, p in enumerate(probs)]
    ref = [_alone(p, [F], precision)[0] for p, F in zip(probs, Fs)]
    solvers = [vasmg.Solver(p, precision=precision, max_ctas=64) for p in probs]
    try:
        # a repeated handle must run in two different groups
        hs = [s.h for s in solvers] + [solvers[0].h]
        Fb = Fs + [Fs[0]]
        Us = [np.zeros_like(F) for F in Fb]
        rc, sts = vasmg.vasmg_solve_batch(hs, Fb, Us, 1e-6)
        assert rc == 0
        for i, (U, st) in enumerate(zip(Us, sts)):
            Ur, itr = ref[i % len(probs)]
            assert st.iterations == itr
            assert _rel(U, Ur) <= 1e-12
    finally:
        for s in solvers:
            s.close()


@pytest.mark.parametrize("batch", [False, True])
def test_server_mix_equals_alone(built, batch):
    """Each request's results equal its solves alone, whether a slot solves
    its own right-hand sides (together, vasmg_solve_multi) or one executor
    solves every ready request's next right-hand side in one batched round
    (vasmg_solve_batch, one launch per level and phase)."""
    probs = [meshgen.make_problem(None, **kw) for kw in MIX]
    nrhs = [1, 3, 2, 1, 2]
    Fss = [_rhs(p, k, 200 + i) for i, (p, k) in enumerate(zip(probs, nrhs))]
    # the server sets its handles up with the lanes per row by rule
    ref = [_alone(p, Fs, "fp32", autotune=False) for p, Fs in zip(probs, Fss)]
    srv = vasmg.Server(slots=3, precision="fp32", batch=batch)
    try:
        tickets, outs = [], []
        for p, Fs in zip(probs, Fss):
            Us = [np.zeros_like(F) for F in Fs]
            outs.append(Us)
            tickets.append(srv.submit(p, Fs, Us))
        stats = [srv.poll(t, -1) for t in tickets]
        for i, st in enumerate(stats):
            assert st is not None and st["status"] == 0
            assert st["n_rhs"] == nrhs[i]
            assert st["latency_ms"] >= st["setup_ms"] + st["solve_ms"] - 1e-6
            assert st["max_rel_res"] < 1e-6
            for U, (Ur, itr) in zip(outs[i], ref[i]):
                assert _rel(U, Ur) <= 1e-12
            assert st["iterations"] == sum(itr for _, itr in ref[i])
        # a released ticket is unknown
        with pytest.raises(vasmg.VasmgError):
            srv.poll(tickets[0], 0)
    finally:
        srv.close()


def test_server_budget_admits_head_alone(built):
    """With a budget smaller than any request, requests run one at a time
    (the head is admitted alone) and still complete correctly."""
    probs = [meshgen.make_problem(None, **kw) for kw in MIX[:3]]
    Fss = [_rhs(p, 1, 300 + i) for i, p in enumerate(probs)]
    ref = [_alone(p, Fs, "fp32", autotune=False) for p, Fs in zip(probs, Fss)]
    srv = vasmg.Server(slots=3, precision="fp32", memory_budget=1)
    try:
        outs = [[np.zeros_like(Fs[0])] for Fs in Fss]
        tickets = [srv.submit(p, Fs, Us) for p, Fs, Us in zip(probs, Fss, outs)]
        stats = [srv.poll(t, -1) for t in tickets]
        for i, st in enumerate(stats):
            assert st["status"] == 0 and st["footprint_bytes"] > 1
            assert _rel(outs[i][0], ref[i][0][0]) <= 1e-12
        # one at a time: each later request waited at least for the earlier one's setup and solve
        for a, b in zip(stats, stats[1:]):
            assert b["queue_ms"] >= a["setup_ms"] + a["solve_ms"] - 1.0
    finally:
        srv.close()
