"""The paper's own validation cases on the GPU path, against the oracle on the
same meshes, and against the analytic solutions.

* 2D channel (Sec. 3.2, Table channel_err): the paper's mesh (49 x 9 quads of
  [0, 5] x [-0.5, 0.5] in P2 triangles: 882 elements, 1,881 nodes, 4,262
  dofs), a traction inlet, W = omega H^2 / nu = 0, 2 pi, 10 pi, 20 pi; the
  relative errors e(T/4), e(T/2) of Eq. total_error against Eq. channel_ana.
* 3D pipe (Sec. 3.4): L/R = 15 with a traction inlet, W = omega R^2 / nu =
  0, 8 pi, 40 pi, 80 pi, errors e(T/2) against Eq. pipe_ana (J0 profile); mesh
  convergence at W = 8 pi.
The GPU solutions match the oracle's LU solutions within 1e-8 and their
errors against the analytic fields match the oracle's errors; the trends the
paper reports hold (exact steady solution on P2, error growing with W,
shrinking with h).  The paper's own percentages (other meshes, its linear
tolerance 1e-6) are context, printed by bench.py --workload validation."""
import numpy as np
import pytest

from oracle import boundary, fem
from paper_2009_06725_gb300 import scvs
from synthetic import meshes, workloads
from synthetic.womersley import channel_profile, pipe_profile

from .gpu_util import rel_l2, stack_modal

pytestmark = pytest.mark.gpu


def _gpu_solve(wl, tol=1e-12):
    m = len(wl["omegas"])
    mesh = wl["mesh"]
    with scvs.Solver(tol=tol, max_cycles=2000) as s:
        mid = scvs.scvs_set_mesh(s.ctx, mesh)
        scvs.scvs_set_physics(s.ctx, mid, wl["rho"], wl["mu"])
        scvs.scvs_set_modes(s.ctx, mid, wl["omegas"], wl["g"])
        scvs.scvs_set_neumann(s.ctx, mid, wl["h"])
        rep = scvs.scvs_solve(s.ctx, mid, m)
        u, p = scvs.scvs_get_modal(s.ctx, mid, m, mesh["xyz"].shape[0], mesh["dim"], mesh["n_vertices"])
    assert all(r["status"] == scvs.SCVS_CONVERGED for r in rep), rep
    return u, p


def _oracle_solve(wl):
    mesh = wl["mesh"]
    faces = boundary.boundary_faces(mesh, scvs.SCVS_TAG_NEUMANN)
    load = np.stack([boundary.neumann_load(mesh, faces, wl["h"][k]) for k in range(len(wl["omegas"]))])
    mats = fem.assemble(mesh)
    return mats, fem.solve_modes(mats, dict(wl, load=load))


def _err_t(Ms, u_h, u_ex, omega, t):
    """e(t) of Eq. total_error for one mode: u(t) = Re(u~ e^{j omega t})."""
    ph = np.exp(1j * omega * t)
    return fem.relative_l2_error(Ms, np.real(u_ex * ph), np.real(u_h * ph))


def test_paper_channel_table():
    rho, mu, H, L, hx = 1.0, 0.01, 0.5, 5.0, 1.0
    Ws = np.array([0.0, 2 * np.pi, 10 * np.pi, 20 * np.pi])
    omegas = Ws * (mu / rho) / H ** 2
    wl = workloads.paper_channel(omegas, rho=rho, mu=mu, hx=hx, neumann_tag=scvs.SCVS_TAG_NEUMANN)
    mesh = wl["mesh"]
    assert mesh["conn"].shape[0] == 882 and mesh["xyz"].shape[0] == 1881
    assert 2 * 1881 + mesh["n_vertices"] == 4262
    u, p = _gpu_solve(wl)
    mats, X = _oracle_solve(wl)
    Xg = stack_modal(u, p)
    y = mesh["xyz"][:, 1]
    errs = []
    for k, w in enumerate(omegas):
        assert rel_l2(Xg[k], X[k]) < 1e-8, k
        ex = np.zeros((mesh["xyz"].shape[0], 2), dtype=np.complex128)
        ex[:, 0] = channel_profile(y, w, H, rho, mu, G=hx / L)
        uo, _ = fem.split_fields(mats, X[k])
        T = 2 * np.pi / w if w > 0 else 1.0
        e_g = [_err_t(mats["Ms"], u[k], ex, w, f * T) for f in (0.25, 0.5)]
        e_o = [_err_t(mats["Ms"], uo, ex, w, f * T) for f in (0.25, 0.5)]
        assert np.allclose(e_g, e_o, rtol=1e-5, atol=1e-9), (k, e_g, e_o)
        errs.append(e_g)
    errs = np.array(errs)
    assert errs[0].max() < 1e-8                       # W = 0: the parabola lies in P2
    assert np.all(np.diff(errs[:, 1]) > 0)            # e(T/2) grows with W
    assert errs[1:, 1].max() < 0.05                   # the paper's SCVS errors: 0.031 / 0.46 / 1.8 %


def _pipe_errors(wl, u, Ms):
    mesh = wl["mesh"]
    r = np.hypot(mesh["xyz"][:, 1], mesh["xyz"][:, 2])
    out = []
    for k, w in enumerate(wl["omegas"]):
        ex = np.zeros((mesh["xyz"].shape[0], 3), dtype=np.complex128)
        ex[:, 0] = pipe_profile(r, w, 1.0, wl["rho"], wl["mu"], G=wl["hx"] / 15.0)
        T = 2 * np.pi / w if w > 0 else 1.0
        out.append(_err_t(Ms, u[k], ex, w, 0.5 * T))
    return np.array(out)


def test_paper_pipe_against_oracle_and_analytic():
    rho, mu = 1.0, 1.0
    Ws = np.array([0.0, 8 * np.pi, 40 * np.pi, 80 * np.pi])
    wl = workloads.traction_inlet(meshes.pipe3d(radius=1.0, length=15.0, n_c=3, n_r=2, n_x=30, jitter=0.0),
                                  Ws * mu / rho, 1.0, rho, mu, scvs.SCVS_TAG_NEUMANN)
    u, p = _gpu_solve(wl)
    mats, X = _oracle_solve(wl)
    Xg = stack_modal(u, p)
    for k in range(len(Ws)):
        assert rel_l2(Xg[k], X[k]) < 1e-8, k
    uo = np.stack([fem.split_fields(mats, X[k])[0] for k in range(len(Ws))])
    e_g, e_o = _pipe_errors(wl, u, mats["Ms"]), _pipe_errors(wl, uo, mats["Ms"])
    assert np.allclose(e_g, e_o, rtol=1e-5, atol=1e-9), (e_g, e_o)
    assert np.all(np.diff(e_g[1:]) > 0), e_g          # error grows with W (Fig. cylinder_msh_freq)


def test_paper_pipe_mesh_convergence():
    """e(T/2) at W = 8 pi shrinks under refinement (GPU only: meshes of 5k-45k nodes)."""
    rho, mu = 1.0, 1.0
    errs = []
    for n_c, n_r, n_x in ((3, 2, 20), (5, 3, 34), (7, 5, 48)):
        wl = workloads.traction_inlet(meshes.pipe3d(radius=1.0, length=15.0, n_c=n_c, n_r=n_r, n_x=n_x, jitter=0.0),
                                      np.array([8 * np.pi * mu / rho]), 1.0, rho, mu, scvs.SCVS_TAG_NEUMANN)
        u, p = _gpu_solve(wl, tol=1e-10)
        Ms = fem.assemble(wl["mesh"])["Ms"]
        errs.append(_pipe_errors(wl, u, Ms)[0])
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[0] / errs[2] > 3.0, errs
