"""Curved (isoparametric) P2 elements on the GPU against the oracle.

Boundary edge nodes projected onto curved walls (Sec. 3.1) make the
elements next to the wall isoparametric; the library integrates them by
quadrature of the quadratic geometry map (the straight ones keep the exact
reference tables).  Compared with the oracle on the same meshes: the
assembled values (1e-12), the all-modes operator through CSR and matrix-free
(1e-12 FP64, 1e-5 FP32), solves (1e-10 FP64, 1e-8 mixed), the curved
channel's exact flow, and the paper's diverging nozzle (Sec. 3.3)."""
import numpy as np
import pytest

from oracle import boundary, fem
from paper_2009_06725_gb300 import scvs
from synthetic import meshes, workloads

from .gpu_util import apply_gpu, open_workload, rel_err, rel_l2, solve, stack_modal

pytestmark = pytest.mark.gpu


def _annulus_workload():
    m = meshes.annulus2d(n_r=3, n_t=12)
    dn = workloads.dirichlet_nodes(m["tag"])
    rng = np.random.default_rng(4)
    omegas = 2 * np.pi * np.arange(4)
    g = (rng.standard_normal((4, dn.size, 2)) + 1j * rng.standard_normal((4, dn.size, 2))) * 0.1
    return dict(mesh=m, omegas=omegas, rho=1.0, mu=0.05, dir_nodes=dn, g=g)


CASES = {
    "annulus": _annulus_workload,
    "curved_pipe": lambda: workloads.pipe_workload(n_c=3, n_r=2, n_x=5, n_modes=4, length=2.5, curved=True),
    "curved_stenosed_pipe": lambda: workloads.pipe_workload(n_c=3, n_r=2, n_x=8, n_modes=3, length=4.0, curved=True,
                                                            stenosis=0.4),
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    wl = CASES[request.param]()
    m = wl["mesh"]
    assert fem.curved_elements(m["xyz"], m["conn"].astype(np.int64), m["dim"]).any()
    return request.param, wl, fem.assemble(m)


def test_curved_values_match_oracle(case):
    _, wl, mats = case
    d = wl["mesh"]["dim"]
    s, mid = open_workload(wl)
    with s:
        v = scvs.scvs_get_values(s.ctx, mid, scvs.SCVS_CSR_S, d)
        assert rel_err(v[0], mats["Ms"].data) < 1e-12
        assert rel_err(v[1], mats["Ks"].data) < 1e-12
        v = scvs.scvs_get_values(s.ctx, mid, scvs.SCVS_CSR_G, d)
        for c in range(d):
            assert rel_err(v[c], mats["D"][c].data) < 1e-12
        v = scvs.scvs_get_values(s.ctx, mid, scvs.SCVS_CSR_GT, d)
        for c in range(d):
            DT = mats["D"][c].T.tocsr()
            DT.sort_indices()
            assert rel_err(v[c], DT.data) < 1e-12


@pytest.mark.parametrize("precision,tol", [(scvs.SCVS_PREC_FP64, 1e-12), (scvs.SCVS_PREC_MIXED, 1e-5)])
@pytest.mark.parametrize("matfree", [False, True])
def test_curved_operator_matches_oracle(case, precision, tol, matfree):
    _, wl, mats = case
    n = fem.dof_count(mats)
    m = len(wl["omegas"])
    X = workloads.random_block(n, m, seed=12)
    Y = fem.masked_apply(mats, wl["omegas"], wl["rho"], wl["mu"], wl["dir_nodes"], X)
    s, mid = open_workload(wl)
    with s:
        Yg = apply_gpu(s, mid, X, precision, matfree=matfree)
    for k in range(m):
        assert rel_err(Yg[:, k], Y[:, k]) < tol, (k, rel_err(Yg[:, k], Y[:, k]))


@pytest.mark.parametrize("precision,solve_tol,err_tol", [(scvs.SCVS_PREC_FP64, 1e-13, 1e-10),
                                                         (scvs.SCVS_PREC_MIXED, 1e-12, 1e-8)])
def test_curved_solve_matches_oracle(case, precision, solve_tol, err_tol):
    _, wl, mats = case
    X = fem.solve_modes(mats, wl)
    s, mid, rep, u, p = solve(wl, precision=precision, tol=solve_tol, max_cycles=2000)
    with s:
        Xg = stack_modal(u, p)
    for k, r in enumerate(rep):
        assert r["status"] == scvs.SCVS_CONVERGED, (k, r)
        assert rel_l2(Xg[k], X[k]) < err_tol, (k, rel_l2(Xg[k], X[k]))


def _neumann_solve(wl, tol=1e-12):
    mesh = wl["mesh"]
    m = len(wl["omegas"])
    with scvs.Solver(tol=tol, max_cycles=2000) as s:
        mid = scvs.scvs_set_mesh(s.ctx, mesh)
        scvs.scvs_set_physics(s.ctx, mid, wl["rho"], wl["mu"])
        scvs.scvs_set_modes(s.ctx, mid, wl["omegas"], wl["g"])
        scvs.scvs_set_neumann(s.ctx, mid, wl["h"])
        rep = scvs.scvs_solve(s.ctx, mid, m)
        u, p = scvs.scvs_get_modal(s.ctx, mid, m, mesh["xyz"].shape[0], mesh["dim"], mesh["n_vertices"])
    assert all(r["status"] == scvs.SCVS_CONVERGED for r in rep), rep
    faces = boundary.boundary_faces(mesh, scvs.SCVS_TAG_NEUMANN)
    load = np.stack([boundary.neumann_load(mesh, faces, wl["h"][k]) for k in range(m)])
    mats = fem.assemble(mesh)
    X = fem.solve_modes(mats, dict(wl, load=load))
    return u, p, mats, X


def test_curved_channel_exact_flow():
    """The exact r ln r flow of the curved channel: GPU = oracle, and third-order convergence."""
    errs = []
    for n in (2, 4, 8):
        wl, uex = workloads.curved_channel(n, 4 * n, neumann_tag=scvs.SCVS_TAG_NEUMANN)
        u, p, mats, X = _neumann_solve(wl)
        assert rel_l2(stack_modal(u, p)[0], X[0]) < 1e-8
        errs.append(fem.relative_l2_error(mats["Ms"], uex, u[0]))
    assert errs[0] / errs[1] > 8.0 and errs[1] / errs[2] > 8.0, errs


def test_paper_nozzle():
    """The paper's diverging nozzle (Sec. 3.3): expansion ratio 2, 600 P2
    triangles and 1,281 nodes with the wall nodes on the curved wall, a zero-mean
    traction inlet with |h_i| ~ omega_i^-2, modes 1..5 (W = omega H^2 / nu up to
    10 pi).  GPU = oracle per mode; the outlet flow rate of the series truncated
    after 1, 3, 5 modes approaches the 10-mode one (the paper reports 25 %, 5.0 %
    and 1.5 % against its 10-mode reference)."""
    nu, H, T = 1.0, 1.0, 1.0
    om1 = 2 * np.pi / T
    mesh = meshes.nozzle2d()
    assert mesh["conn"].shape[0] == 600 and mesh["xyz"].shape[0] == 1281
    assert fem.curved_elements(mesh["xyz"], mesh["conn"].astype(np.int64), 2).sum() > 0
    ks = np.arange(1, 11)
    rng = np.random.default_rng(7)
    amp = ks ** -2.0 * np.exp(2j * np.pi * rng.random(ks.size))  # h_x = Re sum_k amp_k e^{j omega_k t}
    wl = workloads.traction_inlet(mesh, om1 * ks, 1.0, 1.0, nu, scvs.SCVS_TAG_NEUMANN)
    wl["h"] = wl["h"] * amp[:, None, None]
    assert abs(om1 * 5 * H ** 2 / nu - 10 * np.pi) < 1e-12  # W = 2 pi .. 10 pi over modes 1..5, as in the paper
    u, p, mats, X = _neumann_solve(wl)
    Xg = stack_modal(u, p)
    for k in range(ks.size):
        assert rel_l2(Xg[k], X[k]) < 1e-8, k
    # outlet flow rate of every mode: Q_k = int u_x dy over the outlet (P2 trace: Simpson on each edge)
    xyz = mesh["xyz"]
    out = np.flatnonzero(np.abs(xyz[:, 0] - mesh["length"]) < 1e-12)
    o = out[np.argsort(xyz[out, 1])]
    ys = xyz[o, 1]
    Qk = np.array([np.sum((ys[2::2] - ys[:-2:2]) / 6.0 * (u[k][o[:-2:2], 0] + 4 * u[k][o[1::2], 0] + u[k][o[2::2], 0]))
                   for k in range(ks.size)])
    ts = np.linspace(0.0, T, 65)[:-1]
    Q = lambda n: np.real(np.exp(1j * om1 * np.outer(ts, ks[:n])) @ Qk[:n])
    ref = Q(10)
    e = [np.linalg.norm(Q(n) - ref) / np.linalg.norm(ref) for n in (1, 3, 5)]
    assert e[0] > e[1] > e[2] and e[2] < 0.05, e  # oracle on the CPU: 13.8 %, 2.0 %, 0.67 %


def test_curved_traction_pipe_matches_oracle():
    """Traction inlet meeting a curved (projected) wall: the inlet faces along the
    wall are curved and integrated isoparametrically on both sides; the lifted
    right-hand side and the solutions match the oracle."""
    from .test_gpu_parity import _device_view
    mesh = meshes.pipe3d(radius=1.0, length=6.0, n_c=3, n_r=2, n_x=10, jitter=0.0, curved=True)
    wl = workloads.traction_inlet(mesh, np.array([0.0, 8 * np.pi, 40 * np.pi]), 1.0, 1.0, 1.0,
                                  scvs.SCVS_TAG_NEUMANN)
    faces = boundary.boundary_faces(wl["mesh"], scvs.SCVS_TAG_NEUMANN)
    assert boundary.curved_faces(wl["mesh"], faces).any()
    u, p, mats, X = _neumann_solve(wl)
    Xg = stack_modal(u, p)
    for k in range(3):
        assert rel_l2(Xg[k], X[k]) < 1e-8, k
    load = np.stack([boundary.neumann_load(wl["mesh"], faces, wl["h"][k]) for k in range(3)])
    B = fem.rhs_block(mats, dict(wl, load=load))
    with scvs.Solver() as s:
        mid = scvs.scvs_set_mesh(s.ctx, wl["mesh"])
        scvs.scvs_set_physics(s.ctx, mid, wl["rho"], wl["mu"])
        scvs.scvs_set_modes(s.ctx, mid, wl["omegas"], wl["g"])
        scvs.scvs_set_neumann(s.ctx, mid, wl["h"])
        ld = scvs.scvs_mode_stride(s.ctx, mid)
        n = fem.dof_count(mats)
        Bg = _device_view(scvs.scvs_rhs_dev(s.ctx, mid), n * ld).reshape(n, ld)
    for k in range(3):
        assert rel_err(Bg[:, k], B[:, k]) < 1e-13, k
