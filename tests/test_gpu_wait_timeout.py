"""Failure detection without a GPU fault: the bounded device wait.

The sweep kernels wait for neighbouring regions' stage words with an
iteration limit; a wait that runs out raises the abort flag, every CTA
returns, and the solve reports VASMG_ERR_TIMEOUT.  vasmg_probe_wait_timeout
runs that same wait in one CTA against a word that nothing publishes: the
call must return VASMG_ERR_TIMEOUT after a bounded time, and the context must
stay usable (a solve right after it succeeds).
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2505_09064_gb300 import meshgen, vasmg  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def built():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)
    return True


def test_wait_runs_out_and_context_survives(built):
    rc, ms = vasmg.vasmg_probe_wait_timeout()
    assert rc == vasmg.VASMG_ERR_TIMEOUT
    assert 1.0 < ms < 10000.0
    prob = meshgen.make_problem(None, dim=2, n=64, jitter=0.2, seed=3)
    s = vasmg.Solver(prob, precision="fp32", stream=torch.cuda.current_stream().cuda_stream)
    try:
        F = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        s.assemble_load(prob["body_force"], F)
        U = torch.zeros_like(F)
        rc2, st, _ = s.solve(F, U, 1e-6)
        assert rc2 == 0 and st.rel_res < 1e-6 and np.isfinite(U.cpu().numpy()).all()
    finally:
        s.close()
