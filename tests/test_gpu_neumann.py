"""Neumann (traction) inlets on the GPU (scvs_set_neumann) against the oracle:
the lifted right-hand side with the boundary term element by element, the
solutions of the paper's channel with a traction inlet (Sec. 4.1; exact
parabola at omega = 0, Eq. channel_ana) and of a pipe with a traction inlet."""
import numpy as np
import pytest

from oracle import boundary, fem
from paper_2009_06725_gb300 import scvs
from synthetic import meshes, workloads

from .gpu_util import rel_err, rel_l2, stack_modal
from .test_gpu_parity import _device_view

pytestmark = pytest.mark.gpu


def _traction_case(mesh, omegas, hx, rho=1.0, mu=0.01):
    """Inlet nodes become traction nodes (walls stay Dirichlet); h = (hx, 0[, 0])."""
    tag = mesh["tag"].copy()
    inl = (tag & meshes.INLET) != 0
    tag[inl] = (tag[inl] & ~np.uint8(meshes.INLET)) | np.uint8(scvs.SCVS_TAG_NEUMANN)
    mesh = dict(mesh, tag=tag)
    d = mesh["dim"]
    walls = np.flatnonzero((tag & meshes.WALL) != 0)
    N = mesh["xyz"].shape[0]
    h = np.zeros((len(omegas), N, d), dtype=np.complex128)
    h[:, :, 0] = hx
    faces = boundary.boundary_faces(mesh, scvs.SCVS_TAG_NEUMANN)
    load = np.stack([boundary.neumann_load(mesh, faces, h[k]) for k in range(len(omegas))])
    wl = dict(mesh=mesh, omegas=np.asarray(omegas, dtype=np.float64), rho=rho, mu=mu, dir_nodes=walls,
              g=np.zeros((len(omegas), walls.size, d), dtype=np.complex128), load=load)
    return wl, h, faces


def _gpu(wl, h, **opts):
    s = scvs.Solver(**opts)
    mid = scvs.scvs_set_mesh(s.ctx, wl["mesh"])
    scvs.scvs_set_physics(s.ctx, mid, wl["rho"], wl["mu"])
    scvs.scvs_set_modes(s.ctx, mid, wl["omegas"], wl["g"])
    nf = scvs.scvs_set_neumann(s.ctx, mid, h)
    return s, mid, nf


def test_rhs_with_traction_matches_oracle():
    mesh = meshes.channel2d(8, 4)
    wl, h, faces = _traction_case(mesh, [0.0, 0.5, 2.0], hx=1.0)
    mats = fem.assemble(wl["mesh"])
    B = fem.rhs_block(mats, wl)
    s, mid, nf = _gpu(wl, h)
    with s:
        assert nf == faces.shape[0] == 4
        ld = scvs.scvs_mode_stride(s.ctx, mid)
        n = fem.dof_count(mats)
        Bg = _device_view(scvs.scvs_rhs_dev(s.ctx, mid), n * ld).reshape(n, ld)
        # the data persist across a physics change (the lift is rebuilt with them)
        scvs.scvs_set_physics(s.ctx, mid, wl["rho"], wl["mu"])
        Bg2 = _device_view(scvs.scvs_rhs_dev(s.ctx, mid), n * ld).reshape(n, ld)
    for k in range(3):
        assert rel_err(Bg[:, k], B[:, k]) < 1e-13
    assert np.array_equal(Bg, Bg2)


def test_traction_channel_solution():
    hx, rho, mu, L, H = 1.0, 1.0, 0.01, 4.0, 0.5
    mesh = meshes.channel2d(16, 8, length=L, half_height=H)
    oms = [0.0, 2 * np.pi * (mu / rho) / H ** 2, 10 * np.pi * (mu / rho) / H ** 2]
    wl, h, _ = _traction_case(mesh, oms, hx=hx, rho=rho, mu=mu)
    mats = fem.assemble(wl["mesh"])
    X = fem.solve_modes(mats, wl)
    s, mid, _ = _gpu(wl, h, tol=1e-12, max_cycles=2000)
    with s:
        rep = scvs.scvs_solve(s.ctx, mid, len(oms))
        u, p = scvs.scvs_get_modal(s.ctx, mid, len(oms), mesh["xyz"].shape[0], 2, mesh["n_vertices"])
    assert all(r["status"] == scvs.SCVS_CONVERGED for r in rep), rep
    Xg = stack_modal(u, p)
    for k in range(len(oms)):
        assert rel_l2(Xg[k], X[k]) < 1e-8, k
    y = mesh["xyz"][:, 1]
    ux = hx / (2 * mu * L) * (H - y) * (H + y)
    assert np.abs(u[0][:, 0] - ux).max() < 1e-8 * ux.max()


def test_traction_pipe_matches_oracle():
    wl0 = workloads.pipe_workload(n_c=3, n_r=2, n_x=6, n_modes=4, length=3.0)
    wl, h, faces = _traction_case(wl0["mesh"], wl0["omegas"], hx=3.0, rho=wl0["rho"], mu=wl0["mu"])
    mats = fem.assemble(wl["mesh"])
    X = fem.solve_modes(mats, wl)
    s, mid, nf = _gpu(wl, h, tol=1e-12, max_cycles=2000)
    with s:
        assert nf == faces.shape[0]
        rep = scvs.scvs_solve(s.ctx, mid, 4)
        u, p = scvs.scvs_get_modal(s.ctx, mid, 4, wl["mesh"]["xyz"].shape[0], 3, wl["mesh"]["n_vertices"])
    assert all(r["status"] == scvs.SCVS_CONVERGED for r in rep), rep
    Xg = stack_modal(u, p)
    for k in range(4):
        assert rel_l2(Xg[k], X[k]) < 1e-8, k


def test_neumann_before_modes_is_a_state_error():
    mesh = meshes.channel2d(4, 2)
    wl, h, _ = _traction_case(mesh, [0.0], hx=1.0)
    with scvs.Solver() as s:
        mid = scvs.scvs_set_mesh(s.ctx, wl["mesh"])
        with pytest.raises(scvs.ScvsError) as e:
            scvs.scvs_set_neumann(s.ctx, mid, h)
        assert e.value.code == scvs.SCVS_ERR_STATE
