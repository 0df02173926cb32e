"""Failure detection of the persistent kernels' bounded grid barrier.

A cooperative launch in which one block never arrives must not hang: the
other blocks' wait runs out after a short poll limit, they record the
time-out and return, the host reads SCVS_ERR_TIMEOUT, and the context stays
usable (the barrier state is reset and a solve that follows converges).  The
missing arrival is made by the test on the host side of the kernel's logic
(a block told to return at once); nothing faults or traps."""
import numpy as np
import pytest

from paper_2009_06725_gb300 import scvs
from synthetic import workloads

from .gpu_util import open_workload

pytestmark = pytest.mark.gpu


def test_barrier_completes_when_every_block_arrives():
    with scvs.Solver() as s:
        rc, passed = scvs.scvs_barrier_selftest(s.ctx, 1 << 16, 8, -1)
        assert rc == scvs.SCVS_OK and passed == 8


def test_missing_block_times_out_and_context_recovers():
    wl = workloads.channel_workload(16, 4, n_modes=4)
    s, mid = open_workload(wl)
    with s:
        for absent in (0, 5):
            rc, passed = scvs.scvs_barrier_selftest(s.ctx, 1 << 14, 8, absent)
            assert rc == scvs.SCVS_ERR_TIMEOUT and passed == 0
            assert "timed out" in scvs.scvs_last_error(s.ctx)
        # the barrier is reset: a full self-test and a solve with persistent kernels pass
        rc, passed = scvs.scvs_barrier_selftest(s.ctx, 1 << 16, 8, -1)
        assert rc == scvs.SCVS_OK and passed == 8
        rep = scvs.scvs_solve(s.ctx, mid, 4)
        assert all(r["status"] == scvs.SCVS_CONVERGED for r in rep)
        with pytest.raises(scvs.ScvsError):
            scvs.scvs_barrier_selftest(s.ctx, 0, 8, -1)
        with pytest.raises(scvs.ScvsError):
            scvs.scvs_barrier_selftest(s.ctx, 1 << 10, 8, 8)
