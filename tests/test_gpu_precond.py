"""The block preconditioner as an operator (scvs_apply_precond, FP32 path).

Pins of the block upper-triangular form [A_u D; 0 S~] against its
definition, with D taken from the oracle's assembly: the pressure part is the
negated Cahouet-Chabard approximation of the block-diagonal form, and the
velocity part is the velocity cycle applied to r_u - D z_p.  Every
preconditioner kind must also drive the solve to the oracle's solution."""
import numpy as np
import pytest

from oracle import fem
from paper_2009_06725_gb300 import scvs
from synthetic import workloads

from .gpu_util import open_workload, padded_block, rel_l2, solve, stack_modal, torch_cuda

pytestmark = pytest.mark.gpu

M = 8


def _apply(s, mid, X):
    torch = torch_cuda()
    ld = scvs.scvs_mode_stride(s.ctx, mid)
    x = torch.from_numpy(padded_block(X, ld)).to(torch.complex64).cuda()
    y = torch.zeros_like(x)
    torch.cuda.synchronize()
    scvs.scvs_apply_precond(s.ctx, mid, x.data_ptr(), y.data_ptr())
    torch.cuda.synchronize()
    return y.cpu().numpy().astype(np.complex128)[:, : X.shape[1]]


@pytest.fixture(scope="module")
def pipe():
    wl = workloads.pipe_workload(n_c=3, n_r=2, n_x=8, n_modes=M, length=4.0)
    return wl, fem.assemble(wl["mesh"])


def _cols_close(A, B, tol):
    for k in range(A.shape[1]):
        assert rel_l2(A[:, k], B[:, k]) < tol, (k, rel_l2(A[:, k], B[:, k]))


def test_precond_is_linear(pipe):
    wl, mats = pipe
    n = fem.dof_count(mats)
    X = workloads.random_block(n, M, seed=1)
    Y = workloads.random_block(n, M, seed=2)
    s, mid = open_workload(wl)
    with s:
        lhs = _apply(s, mid, 0.5 * X + Y)
        rhs = 0.5 * _apply(s, mid, X) + _apply(s, mid, Y)
    _cols_close(lhs, rhs, 1e-5)


def test_triangular_form_against_definition(pipe):
    wl, mats = pipe
    N, P, d = mats["N"], mats["P"], 3
    n = fem.dof_count(mats)
    R = workloads.random_block(n, M, seed=3)
    s_tri, mid_t = open_workload(wl, precond=scvs.SCVS_PC_TRI_PMG)
    s_dia, mid_d = open_workload(wl, precond=scvs.SCVS_PC_BLOCK_PMG)
    with s_tri, s_dia:
        Z = _apply(s_tri, mid_t, R)
        Zd = _apply(s_dia, mid_d, R)
        # pressure first: the Schur approximation carries the minus sign
        _cols_close(Z[d * N:], -Zd[d * N:], 1e-6)
        # velocity: the cycle on r_u - D z_p (D from the oracle; Dirichlet rows keep r_u)
        zp = Z[d * N:]
        Dz = np.zeros((d * N, M), dtype=np.complex128)
        for c in range(d):
            Dz[c::d] = mats["D"][c] @ zp
        Dz[fem.dirichlet_dofs(wl["dir_nodes"], d)] = 0
        R2 = R.copy()
        R2[: d * N] -= Dz
        R2[d * N:] = 0
        Z2 = _apply(s_tri, mid_t, R2)
        assert np.all(Z2[d * N:] == 0)
        _cols_close(Z2[: d * N], Z[: d * N], 1e-5)
        # with no pressure input both forms are the same velocity cycle
        R3 = R.copy()
        R3[d * N:] = 0
        _cols_close(_apply(s_tri, mid_t, R3), _apply(s_dia, mid_d, R3), 1e-6)


@pytest.mark.parametrize("precond", [scvs.SCVS_PC_BLOCK_CHEB, scvs.SCVS_PC_BLOCK_PMG, scvs.SCVS_PC_TRI_PMG])
def test_every_kind_solves_to_the_oracle(pipe, precond):
    wl, mats = pipe
    X = fem.solve_modes(mats, wl)
    s, mid, rep, u, p = solve(wl, precond=precond, max_cycles=2000)
    with s:
        Xg = stack_modal(u, p)
    for k, r in enumerate(rep):
        assert r["status"] == scvs.SCVS_CONVERGED, (k, r)
        assert rel_l2(Xg[k], X[k]) < 1e-6
    assert np.all(fem.relative_residual(mats, wl, Xg) < 1.05e-8)


@pytest.mark.parametrize("precond", [scvs.SCVS_PC_BLOCK_CHEB, scvs.SCVS_PC_BLOCK_PMG, scvs.SCVS_PC_TRI_PMG,
                                     scvs.SCVS_PC_TRI_PMG_CS])
@pytest.mark.parametrize("precision,solve_tol,err_tol", [(scvs.SCVS_PREC_FP64, 1e-13, 1e-10),
                                                         (scvs.SCVS_PREC_MIXED, 1e-12, 1e-8)])
def test_every_kind_at_the_parity_tolerance(pipe, precond, precision, solve_tol, err_tol):
    """Solved to a 1e-13 (FP64) / 1e-12 (mixed) residual, every kind reaches
    the oracle's solution within 1e-10 / 1e-8 relative L2 per mode."""
    wl, mats = pipe
    X = fem.solve_modes(mats, wl)
    s, mid, rep, u, p = solve(wl, precond=precond, precision=precision, tol=solve_tol, max_cycles=4000)
    with s:
        Xg = stack_modal(u, p)
    for k, r in enumerate(rep):
        assert r["status"] == scvs.SCVS_CONVERGED and r["rel_res"] <= solve_tol, (k, r)
        assert rel_l2(Xg[k], X[k]) < err_tol, (k, rel_l2(Xg[k], X[k]))


def test_triangular_needs_fewer_iterations(pipe):
    wl, _ = pipe
    its = {}
    for precond in (scvs.SCVS_PC_BLOCK_PMG, scvs.SCVS_PC_TRI_PMG):
        s, mid, rep, u, p = solve(wl, precond=precond, max_cycles=2000)
        s.close()
        its[precond] = np.mean([r["iterations"] for r in rep])
    assert its[scvs.SCVS_PC_TRI_PMG] < 0.6 * its[scvs.SCVS_PC_BLOCK_PMG], its


def test_precond_bitwise_reproducible_across_contexts(pipe):
    """Two contexts that each build the mesh from scratch apply a bitwise
    identical preconditioner (mesh tables, spectral bounds and every kernel
    of the cycle are deterministic)."""
    wl, mats = pipe
    R = workloads.random_block(fem.dof_count(mats), M, seed=9)
    outs = []
    for _ in range(3):
        s, mid = open_workload(wl, autotune=0)
        with s:
            outs.append(_apply(s, mid, R))
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


def test_diag_kind_against_definition(pipe):
    """BLOCK_DIAG: z_u = r / diag(mu K_s + |omega| rho M_s) on free velocity rows,
    z_u = r on Dirichlet rows, z_p = (mu / diag M_p + j omega rho / diag L_p) r_p
    with the Laplacian term dropped on outlet vertices (p = 0 there)."""
    wl, mats = pipe
    N, P, d = mats["N"], mats["P"], 3
    R = workloads.random_block(fem.dof_count(mats), M, seed=11)
    s, mid = open_workload(wl, precond=scvs.SCVS_PC_BLOCK_DIAG)
    with s:
        Z = _apply(s, mid, R)
    ks, ms = mats["Ks"].diagonal(), mats["Ms"].diagonal()
    mp, lp = fem.p1_diagonals(wl["mesh"])
    dirn = np.zeros(N, dtype=bool)
    dirn[wl["dir_nodes"]] = True
    out = (wl["mesh"]["tag"][:P] & 4) != 0
    ref = np.empty_like(R)
    for k in range(M):
        w = wl["omegas"][k]
        du = np.repeat(wl["mu"] * ks + abs(w) * wl["rho"] * ms, d)
        ref[: d * N, k] = np.where(np.repeat(dirn, d), R[: d * N, k], R[: d * N, k] / du)
        cp = wl["mu"] / mp + 1j * np.where(out, 0.0, w * wl["rho"] / lp)
        ref[d * N:, k] = cp * R[d * N:, k]
    _cols_close(Z, ref, 1e-6)


def test_apply_precond_before_modes_is_a_state_error(pipe):
    wl, mats = pipe
    torch = torch_cuda()
    n = fem.dof_count(mats)
    with scvs.Solver() as s:
        mid = scvs.scvs_set_mesh(s.ctx, wl["mesh"])
        scvs.scvs_set_physics(s.ctx, mid, wl["rho"], wl["mu"])
        x = torch.zeros((n, M), dtype=torch.complex64, device="cuda")
        with pytest.raises(scvs.ScvsError) as e:
            scvs.scvs_apply_precond(s.ctx, mid, x.data_ptr(), x.data_ptr())
        assert e.value.code == scvs.SCVS_ERR_STATE
