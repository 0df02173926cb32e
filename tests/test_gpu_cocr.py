"""COCR (short-recurrence Krylov method for complex symmetric systems) on the
GPU against the oracle.

The saddle operator A_hat(omega_k) is complex symmetric (reading C1), and the
block-diagonal preconditioner kinds are complex symmetric too, so the
conjugate-residual recurrence with the bilinear form x^T y applies.  Solved to
the parity residuals (1e-13 FP64, 1e-12 mixed with FP64 refinement), every
mode must match the oracle's sparse LU solution within 1e-10 / 1e-8, for one
mesh and for a batch of independent components."""
import numpy as np
import pytest

from oracle import fem
from paper_2009_06725_gb300 import scvs
from synthetic import workloads

from .gpu_util import rel_l2, solve, stack_modal

pytestmark = pytest.mark.gpu

M = 8


@pytest.fixture(scope="module")
def pipe():
    wl = workloads.pipe_workload(n_c=3, n_r=2, n_x=8, n_modes=M, length=4.0)
    return wl, fem.assemble(wl["mesh"])


def test_operator_and_preconditioner_are_complex_symmetric(pipe):
    """x^T A y = y^T A x for the oracle's operator (the property COCR needs)."""
    wl, mats = pipe
    n = fem.dof_count(mats)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    y = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    A = fem.saddle_matrix(mats, wl["omegas"][3], wl["rho"], wl["mu"])
    assert abs(x @ (A @ y) - y @ (A @ x)) < 1e-10 * abs(x @ (A @ y))


@pytest.mark.parametrize("precond", [scvs.SCVS_PC_BLOCK_PMG, scvs.SCVS_PC_BLOCK_CHEB])
@pytest.mark.parametrize("precision,solve_tol,err_tol", [(scvs.SCVS_PREC_FP64, 1e-13, 1e-10),
                                                         (scvs.SCVS_PREC_MIXED, 1e-12, 1e-8)])
def test_cocr_solves_to_the_oracle(pipe, precond, precision, solve_tol, err_tol):
    wl, mats = pipe
    X = fem.solve_modes(mats, wl)
    s, mid, rep, u, p = solve(wl, krylov=scvs.SCVS_KRYLOV_COCR, precond=precond, precision=precision,
                              tol=solve_tol, max_cycles=400)
    with s:
        Xg = stack_modal(u, p)
    for k, r in enumerate(rep):
        assert r["status"] == scvs.SCVS_CONVERGED and r["rel_res"] <= solve_tol, (k, r)
        assert r["iterations"] > 0
        assert rel_l2(Xg[k], X[k]) < err_tol, (k, rel_l2(Xg[k], X[k]))
    assert np.all(fem.relative_residual(mats, wl, Xg) < 10 * solve_tol)


def test_cocr_batch_of_components():
    parts = [workloads.pipe_workload(n_c=3, n_r=2, n_x=n_x, n_modes=4, length=L) for n_x, L in ((4, 2.0), (6, 3.0))]
    U = workloads.union_workload(parts)
    with scvs.Solver(krylov=scvs.SCVS_KRYLOV_COCR, precond=scvs.SCVS_PC_BLOCK_PMG, tol=1e-12) as s:
        mid = scvs.scvs_set_mesh(s.ctx, U["mesh"])
        scvs.scvs_set_components(s.ctx, mid, U["n_comp"], U["node_comp"])
        scvs.scvs_set_physics(s.ctx, mid, U["rho"], U["mu"])
        scvs.scvs_set_modes(s.ctx, mid, U["omegas"], U["g"])
        rep = scvs.scvs_solve(s.ctx, mid, U["n_comp"] * 4)
        mesh = U["mesh"]
        u, p = scvs.scvs_get_modal(s.ctx, mid, 4, mesh["xyz"].shape[0], 3, mesh["n_vertices"])
    assert all(r["status"] == scvs.SCVS_CONVERGED for r in rep)
    for i, (wl, mp) in enumerate(zip(parts, U["maps"])):  # union node ids of every part's nodes
        mats = fem.assemble(wl["mesh"])
        X = fem.solve_modes(mats, wl)
        Pi = wl["mesh"]["n_vertices"]
        for k in range(4):
            xi = np.concatenate([u[k][mp].reshape(-1), p[k][mp[:Pi]]])
            assert rel_l2(xi, X[k]) < 1e-8, (i, k, rel_l2(xi, X[k]))


def test_cocr_uses_a_small_workspace(pipe):
    """COCR keeps 7 vectors per system where FGMRES(30) keeps 61: the pool's
    high-water mark of a solve is far smaller."""
    wl, _ = pipe
    highs = {}
    for kr in (scvs.SCVS_KRYLOV_FGMRES, scvs.SCVS_KRYLOV_COCR):
        s, mid, rep, u, p = solve(wl, krylov=kr, precond=scvs.SCVS_PC_BLOCK_PMG)
        with s:
            assert all(r["status"] == scvs.SCVS_CONVERGED for r in rep)
            scvs.scvs_pool_usage(s.ctx, reset_high=True)
            scvs.scvs_solve(s.ctx, mid, M)
            used, high, _ = scvs.scvs_pool_usage(s.ctx)
            highs[kr] = high - used
    assert highs[scvs.SCVS_KRYLOV_COCR] < 0.3 * highs[scvs.SCVS_KRYLOV_FGMRES], highs
