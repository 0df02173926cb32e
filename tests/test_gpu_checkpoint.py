"""Checkpoint / resume on the GPU: a converged run is written to a checkpoint;
a fresh context resumes from it with SCVS_GUESS_CURRENT, so the stored modes
converge at the first true-residual check with their solution unchanged, a
new mode is solved from zero, and a useless initial solution falls back to a
zero start.

These tests stay off until the warm start's first run on a GPU
(SCVS_RUN_PENDING=1 enables them)."""
import os

import numpy as np
import pytest

from paper_2009_06725_gb300 import scvs
from synthetic import workloads

from .gpu_util import solve

pytestmark = pytest.mark.gpu


def _open(wl, omegas, g, **opts):
    s = scvs.Solver(**opts)
    mid = scvs.scvs_set_mesh(s.ctx, wl["mesh"])
    scvs.scvs_set_physics(s.ctx, mid, wl["rho"], wl["mu"])
    scvs.scvs_set_modes(s.ctx, mid, omegas, g)
    return s, mid


def test_resume_reuses_converged_modes(tmp_path):
    wl = workloads.pipe_workload(n_c=3, n_r=2, n_x=5, n_modes=5, length=2.5)
    mesh = wl["mesh"]
    N, P = mesh["xyz"].shape[0], mesh["n_vertices"]
    path = tmp_path / "pipe.ckpt"
    # first run: modes 0..3, checkpointed
    s, mid = _open(wl, wl["omegas"][:4], wl["g"][:4])
    with s:
        rep = scvs.scvs_solve(s.ctx, mid, 4)
        assert all(r["status"] == scvs.SCVS_CONVERGED for r in rep)
        u_ref, p_ref = scvs.scvs_get_modal(s.ctx, mid, 4, N, 3, P)
        scvs.save_checkpoint(s.ctx, mid, mesh, wl["omegas"][:4], rep, s.opts.tol, path, wl["rho"], wl["mu"],
                             wl["g"][:4])
    # resumed run: all five modes, the first four from the checkpoint
    s, mid = _open(wl, wl["omegas"], wl["g"], guess=scvs.SCVS_GUESS_CURRENT)
    with s:
        idx = scvs.resume_from_checkpoint(s.ctx, mid, mesh, wl["omegas"], s.opts.tol, path, wl["rho"], wl["mu"],
                                          wl["g"])
        assert idx.tolist() == [0, 1, 2, 3, -1]
        # other physics: nothing is reused
        assert scvs.resume_from_checkpoint(s.ctx, mid, mesh, wl["omegas"], s.opts.tol, path, wl["rho"],
                                           2 * wl["mu"], wl["g"]).tolist() == [-1] * 5
        idx = scvs.resume_from_checkpoint(s.ctx, mid, mesh, wl["omegas"], s.opts.tol, path, wl["rho"], wl["mu"],
                                          wl["g"])
        rep = scvs.scvs_solve(s.ctx, mid, 5)
        u, p = scvs.scvs_get_modal(s.ctx, mid, 5, N, 3, P)
    assert all(r["status"] == scvs.SCVS_CONVERGED for r in rep)
    assert [r["iterations"] for r in rep[:4]] == [0, 0, 0, 0] and rep[4]["iterations"] > 0
    assert np.array_equal(u[:4], u_ref) and np.array_equal(p[:4], p_ref)


def test_useless_initial_solution_falls_back_to_zero():
    wl = workloads.pipe_workload(n_c=3, n_r=2, n_x=5, n_modes=3, length=2.5)
    mesh = wl["mesh"]
    N, P = mesh["xyz"].shape[0], mesh["n_vertices"]
    s0, mid0, rep0, u0, p0 = solve(wl)
    s0.close()
    s, mid = _open(wl, wl["omegas"], wl["g"], guess=scvs.SCVS_GUESS_CURRENT)
    with s:
        rng = np.random.default_rng(0)
        scvs.scvs_set_solution(s.ctx, mid, 1e3 * rng.standard_normal((3, N, 3)) + 0j, np.zeros((3, P)) + 0j)
        rep = scvs.scvs_solve(s.ctx, mid, 3)
        u, p = scvs.scvs_get_modal(s.ctx, mid, 3, N, 3, P)
    assert all(r["status"] == scvs.SCVS_CONVERGED for r in rep)
    assert all(r["guess_used"] == 0 for r in rep)  # each start was worse than zero and was dropped
    for k in range(3):
        assert np.linalg.norm(u[k] - u0[k]) <= 1e-6 * np.linalg.norm(u0[k])
