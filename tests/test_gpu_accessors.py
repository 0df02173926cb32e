"""The accessor entry points no other test calls: scvs_dirichlet_count,
scvs_modal_dev (the device block of the solution), scvs_mlp_num_params and
scvs_guess_reset."""
import numpy as np
import pytest

from paper_2009_06725_gb300 import scvs
from synthetic import workloads

from .gpu_util import solve, stack_modal
from .test_gpu_parity import _device_view

pytestmark = pytest.mark.gpu


def test_dirichlet_count_and_device_solution():
    wl = workloads.pipe_workload(n_c=3, n_r=2, n_x=4, n_modes=3, length=2.0)
    s, mid, rep, u, p = solve(wl)
    with s:
        assert scvs.scvs_dirichlet_count(s.ctx, mid) == wl["dir_nodes"].size
        ptr, n_dof, ld = scvs.scvs_modal_dev(s.ctx, mid)
        assert ld == scvs.scvs_mode_stride(s.ctx, mid) and ptr
        X = _device_view(ptr, n_dof * ld).reshape(n_dof, ld)
    assert n_dof == wl["mesh"]["xyz"].shape[0] * 3 + wl["mesh"]["n_vertices"]
    assert np.array_equal(X[:, :3].T, stack_modal(u, p))


def test_mlp_size_and_guess_reset():
    sizes = (5, 32, 32, 32, 8)
    n = sum(a * b + b for a, b in zip(sizes[:-1], sizes[1:]))
    with scvs.Solver() as s:
        scvs.scvs_mlp_init(s.ctx, sizes[0], sizes[1], sizes[-1], np.zeros(n, dtype=np.float32))
        assert scvs.scvs_mlp_num_params(s.ctx) == n
        scvs.scvs_guess_reset(s.ctx)
        assert scvs.scvs_mlp_num_params(s.ctx) == 0
        assert scvs.scvs_guess_info(s.ctx)["n_snapshots"] == 0
