"""CUDA-graph replay of the FGMRES Arnoldi steps: a solve with graphs on
(every step after the first restart cycle replayed from its captured graph)
gives the same solution bit for bit, the same iteration and cycle counts and
the same kernel launch count as plain launches, single mesh and batch."""
import numpy as np
import pytest

from paper_2009_06725_gb300 import scvs
from synthetic import workloads

from .gpu_util import stack_modal

pytestmark = pytest.mark.gpu


def _run(wl, graphs, n_comp=None):
    with scvs.Solver(graphs=graphs, tol=1e-12, max_cycles=2000) as s:
        mid = scvs.scvs_set_mesh(s.ctx, wl["mesh"])
        if n_comp:
            scvs.scvs_set_components(s.ctx, mid, wl["n_comp"], wl["node_comp"])
        scvs.scvs_set_physics(s.ctx, mid, wl["rho"], wl["mu"])
        scvs.scvs_set_modes(s.ctx, mid, wl["omegas"], wl["g"])
        n0 = scvs.scvs_launch_count(s.ctx)
        m = len(wl["omegas"]) * (wl.get("n_comp") or 1)
        rep = scvs.scvs_solve(s.ctx, mid, m)
        launches = scvs.scvs_launch_count(s.ctx) - n0
        mesh = wl["mesh"]
        u, p = scvs.scvs_get_modal(s.ctx, mid, len(wl["omegas"]), mesh["xyz"].shape[0], mesh["dim"],
                                   mesh["n_vertices"])
    return rep, launches, stack_modal(u, p)


@pytest.mark.parametrize("name", ["pipe", "batch"])
def test_graph_replay_is_identical(name):
    if name == "pipe":
        wl, nc = workloads.pipe_workload(n_c=3, n_r=2, n_x=6, n_modes=8, length=3.0), None
    else:
        wl = workloads.union_workload([workloads.pipe_workload(n_c=3, n_r=2, n_x=n, n_modes=4, length=L)
                                       for n, L in ((4, 2.0), (7, 3.5))])
        nc = wl["n_comp"]
    r0, l0, X0 = _run(wl, 0, nc)
    r1, l1, X1 = _run(wl, 1, nc)
    assert max(r["cycles"] for r in r0) >= 2  # later cycles replay graphs
    assert all(r["status"] == scvs.SCVS_CONVERGED for r in r1)
    assert [(r["iterations"], r["cycles"]) for r in r0] == [(r["iterations"], r["cycles"]) for r in r1]
    assert l0 == l1
    assert np.array_equal(X0, X1)
