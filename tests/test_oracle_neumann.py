"""Pins of the Neumann (traction) boundary term of the oracle: face tables,
P2 face mass matrices against closed forms, and the paper's channel case with
a traction inlet (Sec. 4.1) against its analytic solution (Eq. channel_ana):
exact at omega = 0 (the parabola lies in P2), third-order convergent at
W = 2 pi."""
import numpy as np
import pytest

from oracle import boundary, fem
from synthetic import meshes, workloads


def test_face_tables_are_faces():
    # every local face's edge nodes are the midpoints of its vertex pairs (affine P2)
    for mesh in (meshes.channel2d(4, 2), workloads.pipe_workload(n_c=3, n_r=2, n_x=3, n_modes=1)["mesh"]):
        xyz, conn = mesh["xyz"], mesh["conn"]
        local = boundary.FACES_2D if mesh["dim"] == 2 else boundary.FACES_3D
        nv = mesh["dim"]
        pairs = ((0, 1),) if nv == 2 else ((0, 1), (1, 2), (2, 0))
        for f in local:
            for j, (a, b) in enumerate(pairs):
                mid = 0.5 * (xyz[conn[:, f[a]]] + xyz[conn[:, f[b]]])
                assert np.allclose(xyz[conn[:, f[nv + j]]], mid, atol=1e-12)


def test_face_mass_row_sums_closed_form():
    # int over a P2 face of each basis function: segment L/6, L/6, 2L/3;
    # triangle 0 at the vertices and |F|/3 at the edge nodes
    seg = boundary.face_mass_reference(1)
    assert np.allclose(seg.sum(axis=1), [1 / 6, 1 / 6, 2 / 3], atol=1e-15)
    tri = boundary.face_mass_reference(2)
    assert np.allclose(tri.sum(axis=1), [0, 0, 0, 1 / 6, 1 / 6, 1 / 6], atol=1e-15)
    for M in (seg, tri):
        assert np.allclose(M, M.T) and np.all(np.linalg.eigvalsh(M) > 0)


def test_inlet_faces_and_total_measure():
    mesh = meshes.channel2d(8, 4)
    faces = boundary.boundary_faces(mesh, meshes.INLET)
    assert faces.shape == (4, 3)  # one triangle edge per inlet cell
    assert np.allclose(mesh["xyz"][faces.ravel(), 0], 0.0)
    Mg = boundary.face_mass(mesh, faces)
    assert Mg.sum() == pytest.approx(2 * mesh["half_height"], rel=1e-14)
    # with every node tagged only faces of one element count: the whole boundary
    every = dict(mesh, tag=mesh["tag"] | 8)
    allf = boundary.boundary_faces(every, 8)
    assert allf.shape[0] == 2 * (8 + 4)
    assert boundary.face_mass(every, allf).sum() == pytest.approx(2 * (4.0 + 2 * mesh["half_height"]), rel=1e-14)
    wl = workloads.pipe_workload(n_c=6, n_r=4, n_x=3, n_modes=1)
    faces3 = boundary.boundary_faces(wl["mesh"], meshes.INLET)
    assert np.allclose(wl["mesh"]["xyz"][faces3.ravel(), 0], 0.0)
    area = boundary.face_measures(wl["mesh"], faces3).sum()
    assert boundary.face_mass(wl["mesh"], faces3).sum() == pytest.approx(area, rel=1e-13)
    assert abs(area - np.pi) < 0.05 * np.pi  # polygonal unit disk
    # no outlet face is taken for the inlet and vice versa
    out = boundary.boundary_faces(wl["mesh"], meshes.OUTLET)
    assert out.shape[0] == faces3.shape[0]
    assert not set(map(tuple, np.sort(out, axis=1))) & set(map(tuple, np.sort(faces3, axis=1)))


def _traction_channel(nx, ny, omegas, hx=1.0, rho=1.0, mu=0.01, L=4.0, H=0.5):
    mesh = meshes.channel2d(nx, ny, length=L, half_height=H)
    walls = np.flatnonzero((mesh["tag"] & meshes.WALL) != 0)
    faces = boundary.boundary_faces(mesh, meshes.INLET)
    h = np.zeros((mesh["xyz"].shape[0], 2))
    h[:, 0] = hx
    b = boundary.neumann_load(mesh, faces, h)
    wl = dict(mesh=mesh, omegas=np.asarray(omegas, dtype=np.float64), rho=rho, mu=mu, dir_nodes=walls,
              g=np.zeros((len(omegas), walls.size, 2), dtype=np.complex128),
              load=np.stack([b.astype(np.complex128)] * len(omegas)))
    mats = fem.assemble(mesh)
    return mesh, mats, wl, fem.solve_modes(mats, wl)


def test_traction_channel_steady_is_exact():
    hx, mu, L, H = 1.0, 0.01, 4.0, 0.5
    mesh, mats, wl, X = _traction_channel(8, 4, [0.0], hx=hx, mu=mu, L=L, H=H)
    u, p = fem.split_fields(mats, X[0])
    y = mesh["xyz"][:, 1]
    ux = hx / (2 * mu * L) * (H - y) * (H + y)
    assert np.abs(u[:, 0] - ux).max() < 1e-10 * ux.max()
    assert np.abs(u[:, 1]).max() < 1e-10 * ux.max()
    x = mesh["xyz"][: mats["P"], 0]
    assert np.abs(p - hx * (L - x) / L).max() < 1e-10 * hx
    assert np.all(fem.relative_residual(mats, wl, X) < 1e-12)


def test_traction_channel_oscillatory_converges_to_cosh_profile():
    hx, rho, mu, L, H = 1.0, 1.0, 0.01, 4.0, 0.5
    W = 2 * np.pi
    w = W * (mu / rho) / H ** 2
    lam = np.sqrt(1j * W)
    errs = []
    for nx, ny in ((8, 4), (16, 8)):
        mesh, mats, wl, X = _traction_channel(nx, ny, [w], hx=hx, rho=rho, mu=mu, L=L, H=H)
        u, _ = fem.split_fields(mats, X[0])
        y = mesh["xyz"][:, 1]
        ux = -1j * hx / (rho * L * w) * (1 - np.cosh(lam * y / H) / np.cosh(lam))
        ref = np.stack([ux, np.zeros_like(ux)], axis=1)
        errs.append(fem.relative_l2_error(mats["Ms"], ref, u))
    assert errs[0] < 1e-2 and errs[0] / errs[1] > 6.0, errs  # measured 2.5e-3, ratio 11.5


def test_spectral_algorithm_end_to_end_channel():
    """Steps 1-4 of the algorithm of Sec. 3 on the channel of Sec. 4.1: a periodic
    traction with a steady part and two harmonics is sampled in time, transformed
    (Eq. SCVS_bc), truncated where e_M vanishes (Eq. mode_error), every mode is
    solved with its Neumann load, and the reconstruction (Eq. sol_reconstruct)
    matches the analytic u_x(y, t) = Re sum_k u~_k(y) e^{j omega_k t} (Eq.
    channel_ana) at the samples."""
    from oracle import bcspec
    rho, mu, L, H, T, n_t = 1.0, 0.01, 4.0, 0.5, 1.0, 16
    amp = {0: 0.5, 1: 0.3 * np.exp(0.4j), 2: 0.1 * np.exp(-1.1j)}  # h_x = Re sum_k amp_k e^{j omega_k t}
    t = np.arange(n_t) * T / n_t
    hx_t = sum(np.real(a * np.exp(2j * np.pi * k * t / T)) for k, a in amp.items())
    # steps 1-2: spectrum and the number of modes from the a priori error
    N_m, e2 = bcspec.select_modes([(hx_t[:, None], np.ones(1))], 1e-12, 6)
    assert N_m == 2
    c = bcspec.solver_modes(bcspec.fourier_coefficients(hx_t, N_m + 1))
    assert np.allclose(c, [amp[0], amp[1], amp[2]], atol=1e-14)
    # step 3: one Neumann solve per mode (nodal traction c_k on the inlet)
    omegas = 2 * np.pi * np.arange(N_m + 1) / T
    mesh = meshes.channel2d(32, 16, length=L, half_height=H)
    walls = np.flatnonzero((mesh["tag"] & meshes.WALL) != 0)
    faces = boundary.boundary_faces(mesh, meshes.INLET)
    N = mesh["xyz"].shape[0]
    unit = np.zeros((N, 2))
    unit[:, 0] = 1.0
    b1 = boundary.neumann_load(mesh, faces, unit)
    wl = dict(mesh=mesh, omegas=omegas, rho=rho, mu=mu, dir_nodes=walls,
              g=np.zeros((N_m + 1, walls.size, 2), dtype=np.complex128),
              load=np.stack([ck * b1 for ck in c]))
    mats = fem.assemble(mesh)
    X = fem.solve_modes(mats, wl)
    U = np.stack([fem.split_fields(mats, X[k])[0] for k in range(N_m + 1)])
    # step 4: reconstruction against the analytic solution in time
    u_t = fem.reconstruct(U, omegas, n_t, T)
    y = mesh["xyz"][:, 1]
    ref = np.zeros((N_m + 1, N, 2), dtype=np.complex128)
    for k, w in enumerate(omegas):
        if w == 0:
            ref[k, :, 0] = c[k] / (2 * mu * L) * (H - y) * (H + y)
        else:
            lam = np.sqrt(1j * w * H ** 2 * rho / mu)
            ref[k, :, 0] = -1j * c[k] / (rho * L * w) * (1 - np.cosh(lam * y / H) / np.cosh(lam))
    ref_t = fem.reconstruct(ref, omegas, n_t, T)
    errs = [fem.relative_l2_error(mats["Ms"], ref_t[s], u_t[s]) for s in range(n_t)]
    assert max(errs) < 1e-4, max(errs)  # measured 1.5e-5 on the 32x16 mesh (harmonics at W = 50 pi, 100 pi)


def test_curved_face_mass_closed_forms():
    """A P2 segment whose midpoint is displaced by delta: sum M_F = arc length of
    x(t) = t L + 4 delta t (1 - t) n, i.e. (1/(4 delta)) [s/2 sqrt(L^2+s^2) + L^2/2 ln(s + sqrt(L^2+s^2))]
    from 0 to 4 delta (closed form); a planar triangle face with one curved edge:
    area |T| + (2/3) |chord| delta; straight faces keep the reference matrices."""
    import math
    L, delta = 2.0, 0.3
    xyz = np.array([[0.0, 0.0], [L, 0.0], [0.5 * L, delta]])
    m2 = dict(xyz=xyz, dim=2)
    faces = np.array([[0, 1, 2]])
    assert boundary.curved_faces(m2, faces).all()
    s4 = 4 * delta
    F = lambda s: 0.5 * s * math.sqrt(L * L + s * s) + 0.5 * L * L * math.log(s + math.sqrt(L * L + s * s))
    arc = (F(s4) - F(0.0)) / (4 * delta)
    Mf = boundary.face_mass_iso(m2, faces)[0]
    assert abs(Mf.sum() - arc) < 1e-7 * arc       # sqrt integrand: 6.9e-9 quadrature error at delta / L = 0.15
    assert np.allclose(Mf, Mf.T, atol=1e-15)
    # planar face in 3D (z = 0) with the edge node of edge (0,1) displaced in-plane
    x3 = np.array([[0, 0, 0], [2, 0, 0], [0, 1, 0], [1, -delta, 0], [1, 0.5, 0], [0, 0.5, 0]], dtype=float)
    f3 = np.array([[0, 1, 2, 3, 4, 5]])
    m3 = dict(xyz=x3, dim=3)
    assert abs(boundary.face_mass_iso(m3, f3)[0].sum() - (1.0 + (2.0 / 3.0) * 2.0 * delta)) < 1e-13
    # straight faces: the isoparametric rule gives the closed-form matrices
    x3s = x3.copy()
    x3s[3] = [1, 0, 0]
    ms = dict(xyz=x3s, dim=3)
    assert not boundary.curved_faces(ms, f3).any()
    ref = boundary.face_measures(ms, f3)[0] / 0.5 * boundary.face_mass_reference(2)
    assert np.abs(boundary.face_mass_iso(ms, f3)[0] - ref).max() < 1e-15
