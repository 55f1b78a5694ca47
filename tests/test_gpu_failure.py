"""Failure detection without a GPU fault: the persistent kernels' grid barrier
waits are bounded.  A block that never arrives makes the others' waits run out;
they record QP_TIMEOUT and return, and the context stays usable."""
import numpy as np
import pytest
import torch

from paper_1808_02558_gb300 import binding, workload
from synth import scene_for

pytestmark = pytest.mark.gpu


def test_barrier_wait_runs_out_and_context_survives():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = binding.Context()
    # about 1 ms of clock ticks: the absent block's peers give up quickly
    assert c.selftest_barrier(2_000_000, absent_block=3) == binding.QP_TIMEOUT
    assert c.selftest_barrier(2_000_000, absent_block=-1) == binding.QP_OK
    # the same context still assembles and solves
    s = scene_for("pile8", 1)
    _, con = workload.assemble(c, s)
    g = torch.zeros(con.P, dtype=torch.float64, device="cuda")
    lam = torch.zeros(2 * con.Nc, dtype=torch.float64, device="cuda")
    st = c.state(g, lam)
    c.pdip_init(st, 1.0)
    rhs = torch.empty(con.P, dtype=torch.float64, device="cuda")
    c.newton_rhs(st, rhs)
    dx = torch.empty_like(rhs)
    stats = c.newton_solve(st, rhs, dx, c.solve_opts(tol=1e-10), allow=())
    assert stats.status == binding.QP_OK and np.isfinite(stats.rel_res) and stats.rel_res <= 1e-10
    with pytest.raises(binding.QPError):
        c.selftest_barrier(0, absent_block=1)
    c.close()
