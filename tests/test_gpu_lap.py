"""Two-level pressure Laplacian of the Schur approximation (opts.lap_size).

Pins:
* the coarse level's aggregates are a valid partition of the vertices off the
  outlet: -1 exactly on the outlet vertices, every aggregate non-empty and
  connected in the vertex graph without them, at most 1024 per component;
* the preconditioner's pressure block, as an operator, equals its definition
  written out here with the oracle's P1 matrices and the library's spectral
  bounds and aggregates.  Block-diagonal form: z_p = mu pM(r) + j omega rho B r
  with pM the degree-4 Chebyshev-Jacobi polynomial of M_p on
  [lam_m / 6, 1.1 lam_m] and B the two-level cycle
      x1 = S r,  x2 = x1 + R (R^T L R)^-1 R^T (r - L x1),  B r = x2 + S (r - L x2),
  S the lap_smooth-step Chebyshev-Jacobi polynomial of L (the P1 Laplacian
  with p = 0 on the outlet) on [lam_l / 120, 1.1 lam_l], R the aggregates'
  indicator;
* B is symmetric (a requirement of COCR's preconditioner);
* solves with the cycle (other aggregate counts and degrees too) and with the
  plain polynomial reach the oracle's solutions;
* a batch with a component whose outlet is tagged as a traction boundary
  instead (no vertex with p = 0 there, so L is singular) keeps the plain
  polynomial and still solves."""
from collections import deque

import numpy as np
import pytest

from oracle import fem
from paper_2009_06725_gb300 import scvs
from synthetic import meshes, workloads

from .gpu_util import open_workload, padded_block, rel_l2, solve, stack_modal, torch_cuda
from .test_aggregates_cpu import vertex_graph

pytestmark = pytest.mark.gpu

M = 8


def _cases():
    return {
        "pipe": workloads.pipe_workload(n_c=3, n_r=2, n_x=8, n_modes=M, length=4.0),
        "channel": workloads.channel_workload(24, 6, n_modes=M),
    }


@pytest.fixture(scope="module", params=["pipe", "channel"])
def case(request):
    return request.param, _cases()[request.param]


def _apply(s, mid, X):
    torch = torch_cuda()
    ld = scvs.scvs_mode_stride(s.ctx, mid)
    x = torch.from_numpy(padded_block(X, ld)).to(torch.complex64).cuda()
    y = torch.zeros_like(x)
    torch.cuda.synchronize()
    scvs.scvs_apply_precond(s.ctx, mid, x.data_ptr(), y.data_ptr())
    torch.cuda.synchronize()
    return y.cpu().numpy().astype(np.complex128)[:, : X.shape[1]]


def _cheb_seq(lo, hi, s):
    """inv_theta and the (alpha_i, beta_i) of the three-term Chebyshev recurrence."""
    th, de = 0.5 * (hi + lo), 0.5 * (hi - lo)
    sg = th / de
    rho_prev = 1.0 / sg
    al, be = np.zeros(s), np.zeros(s)
    for i in range(1, s):
        rho = 1.0 / (2.0 * sg - rho_prev)
        al[i], be[i] = rho * rho_prev, 2.0 * rho / de
        rho_prev = rho
    return 1.0 / th, al, be


def _cheb(A, r, lo, hi, s):
    """s Chebyshev-Jacobi steps for A z = r from z = 0."""
    inv_th, al, be = _cheb_seq(lo, hi, s)
    dinv = 1.0 / A.diagonal()[:, None]
    z_prev = np.zeros_like(r)
    z = inv_th * dinv * r
    for i in range(1, s):
        z, z_prev = z + al[i] * (z - z_prev) + be[i] * dinv * (r - A @ z), z
    return z


def _outlet(mesh):
    P = mesh["n_vertices"]
    return (mesh["tag"][:P] & meshes.OUTLET) != 0


def test_aggregates_partition_the_vertices_off_the_outlet(case):
    name, wl = case
    mesh = wl["mesh"]
    P = mesh["n_vertices"]
    s, mid = open_workload(wl, precond=scvs.SCVS_PC_BLOCK_PMG)
    with s:
        _apply(s, mid, workloads.random_block(fem.dof_count(fem.assemble(mesh)), M, seed=1))
        info = scvs.scvs_lap_info(s.ctx, mid, P)
    out = _outlet(mesh)
    agg = info["agg"]
    assert info["on"] == 1 and info["unanchored"] == 0 and info["singular"] == 0, info
    assert info["n_blk"] == 1 and 1 <= info["na_max"] <= 1024 and info["n_agg"] == info["na_max"]
    assert np.array_equal(agg < 0, out)
    assert set(np.unique(agg[~out])) == set(range(info["n_agg"]))
    ptr, col = vertex_graph(mesh)
    for a in range(info["n_agg"]):
        members = np.flatnonzero(agg == a)
        seen = {members[0]}
        todo = deque([members[0]])
        while todo:
            v = todo.popleft()
            for u in col[ptr[v]:ptr[v + 1]]:
                if agg[u] == a and u not in seen:
                    seen.add(u)
                    todo.append(u)
        assert len(seen) == members.size, (a, len(seen), members.size)


@pytest.mark.parametrize("lap_size,lap_smooth", [(0, 0), (3, 3), (60, 5)])
def test_pressure_block_against_definition(case, lap_size, lap_smooth):
    name, wl = case
    mesh = wl["mesh"]
    mats = fem.assemble(mesh)
    N, P, d = mats["N"], mats["P"], mesh["dim"]
    n = fem.dof_count(mats)
    rng = np.random.default_rng(7)
    R = np.zeros((n, M), dtype=np.complex128)
    R[d * N:] = rng.standard_normal((P, M)) + 1j * rng.standard_normal((P, M))
    s, mid = open_workload(wl, precond=scvs.SCVS_PC_BLOCK_PMG, lap_size=lap_size, lap_smooth=lap_smooth)
    with s:
        Z = _apply(s, mid, R)[d * N:]
        info = scvs.scvs_lap_info(s.ctx, mid, P)
        lam_m, lam_l, _, _ = scvs.scvs_pc_bounds(s.ctx, mid, M)
    assert info["on"] == 1
    deg = lap_smooth or 8
    out = _outlet(mesh)
    F = np.flatnonzero(~out)
    Mp = fem.p1_mass(mesh).tocsr()
    L = fem.p1_stiffness(mesh).tocsr()[F][:, F]
    agg = info["agg"][F]
    Rc = np.zeros((F.size, info["n_agg"]))
    Rc[np.arange(F.size), agg] = 1.0
    Ac_inv = np.linalg.inv(Rc.T @ (L @ Rc))
    rp = R[d * N:]
    zM = _cheb(Mp, rp, lam_m / 6.0, 1.1 * lam_m, 4)
    x1 = _cheb(L, rp[F], lam_l / 120.0, 1.1 * lam_l, deg)
    x2 = x1 + Rc @ (Ac_inv @ (Rc.T @ (rp[F] - L @ x1)))
    x3 = x2 + _cheb(L, rp[F] - L @ x2, lam_l / 120.0, 1.1 * lam_l, deg)
    zL = np.zeros_like(rp)
    zL[F] = x3
    for k in range(M):
        w = wl["omegas"][k] * wl["rho"]
        ref = wl["mu"] * zM[:, k] + 1j * w * zL[:, k]
        assert rel_l2(Z[:, k], ref) < 1e-4, (name, k, rel_l2(Z[:, k], ref))


def test_two_level_cycle_is_symmetric(case):
    name, wl = case
    mesh = wl["mesh"]
    mats = fem.assemble(mesh)
    N, P, d = mats["N"], mats["P"], mesh["dim"]
    n = fem.dof_count(mats)
    rng = np.random.default_rng(11)
    X = np.zeros((n, M), dtype=np.complex128)
    Y = np.zeros((n, M), dtype=np.complex128)
    X[d * N:] = rng.standard_normal((P, M))
    Y[d * N:] = rng.standard_normal((P, M))
    s, mid = open_workload(wl, precond=scvs.SCVS_PC_BLOCK_PMG)
    with s:
        BX = _apply(s, mid, X)[d * N:]
        BY = _apply(s, mid, Y)[d * N:]
    for k in range(1, M):  # real input: the imaginary part is omega rho B r
        w = wl["omegas"][k] * wl["rho"]
        bx, by = BX[:, k].imag / w, BY[:, k].imag / w
        xy, yx = Y[d * N:, k].real @ bx, X[d * N:, k].real @ by
        assert abs(xy - yx) < 1e-5 * np.sqrt(abs((X[d * N:, k].real @ bx) * (Y[d * N:, k].real @ by))), (k, xy, yx)


@pytest.mark.parametrize("lap_size,lap_smooth,precision,tol,err", [
    (0, 0, scvs.SCVS_PREC_MIXED, 1e-8, 1e-6),
    (3, 3, scvs.SCVS_PREC_MIXED, 1e-8, 1e-6),
    (-1, 0, scvs.SCVS_PREC_MIXED, 1e-8, 1e-6),
    (0, 0, scvs.SCVS_PREC_FP64, 1e-12, 1e-10),
])
def test_solves_reach_the_oracle(case, lap_size, lap_smooth, precision, tol, err):
    name, wl = case
    mats = fem.assemble(wl["mesh"])
    X = fem.solve_modes(mats, wl)
    s, mid, rep, u, p = solve(wl, lap_size=lap_size, lap_smooth=lap_smooth, precision=precision, tol=tol,
                              max_cycles=2000)
    with s:
        Xg = stack_modal(u, p)
        info = scvs.scvs_lap_info(s.ctx, mid)
    assert info["on"] == (0 if lap_size < 0 else 1)
    for k, r in enumerate(rep):
        assert r["status"] == scvs.SCVS_CONVERGED, (k, r)
        assert rel_l2(Xg[k], X[k]) < err, (k, rel_l2(Xg[k], X[k]))


def test_component_without_outlet_keeps_the_polynomial():
    """A batch whose second channel has its outlet tagged as a traction
    boundary (zero traction: the same flow, but no vertex with p = 0, so L is
    singular on that component) keeps the plain polynomial for the mesh."""
    a = workloads.channel_workload(24, 6, n_modes=4)
    b = workloads.channel_workload(16, 4, n_modes=4)
    mesh_b = dict(b["mesh"])
    tag = mesh_b["tag"].copy()
    out = (tag & meshes.OUTLET) != 0
    tag[out] = (tag[out] & ~np.uint8(meshes.OUTLET)) | np.uint8(scvs.SCVS_TAG_NEUMANN)
    mesh_b["tag"] = tag
    b = dict(b, mesh=mesh_b)
    U = workloads.union_workload([a, b])
    m = len(U["omegas"])
    with scvs.Solver(max_cycles=2000) as s:
        mid = scvs.scvs_set_mesh(s.ctx, U["mesh"])
        scvs.scvs_set_components(s.ctx, mid, U["n_comp"], U["node_comp"])
        scvs.scvs_set_physics(s.ctx, mid, U["rho"], U["mu"])
        scvs.scvs_set_modes(s.ctx, mid, U["omegas"], U["g"])
        rep = scvs.scvs_solve(s.ctx, mid, U["n_comp"] * m)
        info = scvs.scvs_lap_info(s.ctx, mid, U["mesh"]["n_vertices"])
        N, P = U["mesh"]["xyz"].shape[0], U["mesh"]["n_vertices"]
        u, p = scvs.scvs_get_modal(s.ctx, mid, m, N, 2, P)
    assert info["on"] == 0 and info["unanchored"] == 1 and info["n_blk"] == 2 and np.all(info["agg"] == -1), info
    for i, (wl, mp) in enumerate(zip((a, b), U["maps"])):
        X = fem.solve_modes(fem.assemble(wl["mesh"]), wl)
        Pi = wl["mesh"]["n_vertices"]
        for k in range(m):
            assert rep[i * m + k]["status"] == scvs.SCVS_CONVERGED, (i, k, rep[i * m + k])
            xi = np.concatenate([u[k][mp].reshape(-1), p[k][mp[:Pi]]])
            assert rel_l2(xi, X[k]) < 1e-6, (i, k)
