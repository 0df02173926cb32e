"""Pins of the FP64 oracle against closed forms, invariants and the paper's
exact cases (no GPU).  Each test is chosen so that a plausible slip in the
oracle (a dropped term, a wrong sign or index, a transposed operand) fails it.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import fem
from synthetic import meshes, workloads
from synthetic.womersley import channel_profile, pipe_profile

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------ quadrature

@pytest.mark.parametrize("dim", [2, 3])
def test_simplex_rule_exact_on_monomials(dim):
    """int over the unit simplex of x^a y^b (z^c) = a! b! (c!) / (a+b(+c)+dim)!"""
    pts, w = fem.simplex_rule(dim, 5)
    for a in range(5):
        for b in range(5 - a):
            cs = range(5 - a - b) if dim == 3 else [0]
            for c in cs:
                f = pts[:, 0] ** a * pts[:, 1] ** b * (pts[:, 2] ** c if dim == 3 else 1.0)
                exact = math.factorial(a) * math.factorial(b) * math.factorial(c) / math.factorial(a + b + c + dim)
                assert abs(w @ f - exact) < 1e-15


# ------------------------------------------------------------------ basis

@pytest.mark.parametrize("dim", [2, 3])
def test_p2_basis_nodal_and_partition(dim):
    verts = np.vstack([np.zeros(dim), np.eye(dim)])
    edges = fem._edges(dim)
    nodes = np.vstack([verts] + [0.5 * (verts[i] + verts[j]) for i, j in edges])
    phi, dphi = fem.p2_basis(dim, nodes)
    assert np.allclose(phi, np.eye(nodes.shape[0]), atol=1e-14)
    rng = np.random.default_rng(1)
    x = rng.dirichlet(np.ones(dim + 1), size=20)[:, 1:]
    phi, dphi = fem.p2_basis(dim, x)
    assert np.allclose(phi.sum(axis=1), 1.0)
    assert np.allclose(dphi.sum(axis=1), 0.0, atol=1e-13)
    # reproduces the linear function x_0 exactly
    assert np.allclose(phi @ nodes[:, 0], x[:, 0])
    # gradient check against central differences
    h = 1e-6
    for i in range(dim):
        e = np.zeros(dim)
        e[i] = h
        fd = (fem.p2_basis(dim, x + e)[0] - fem.p2_basis(dim, x - e)[0]) / (2 * h)
        assert np.allclose(fd, dphi[:, :, i], atol=1e-8)


# ------------------------------------------------------- element matrices

def _one_element(dim, seed=0):
    rng = np.random.default_rng(seed)
    v = np.vstack([np.zeros(dim), np.eye(dim)]) + 0.1 * rng.standard_normal((dim + 1, dim))
    if np.linalg.det((v[1:] - v[0]).T) < 0:
        v[[1, 2]] = v[[2, 1]]
    edges = fem._edges(dim)
    xyz = np.vstack([v] + [0.5 * (v[i] + v[j]) for i, j in edges])
    conn = np.arange(xyz.shape[0])[None, :]
    vol = abs(np.linalg.det((v[1:] - v[0]).T)) / math.factorial(dim)
    return xyz, conn, vol


@pytest.mark.parametrize("dim", [2, 3])
def test_element_mass_row_sums_closed_form(dim):
    """int M_A over a straight P2 simplex: triangle 0 (vertex) and |T|/3 (edge);
    tetrahedron -|T|/20 (vertex) and |T|/5 (edge)."""
    xyz, conn, vol = _one_element(dim)
    Me, Ke, De = fem.element_matrices(xyz, conn, dim)
    rs = Me[0].sum(axis=1)
    if dim == 2:
        assert np.allclose(rs[:3], 0.0, atol=1e-15)
        assert np.allclose(rs[3:], vol / 3)
    else:
        assert np.allclose(rs[:4], -vol / 20)
        assert np.allclose(rs[4:], vol / 5)
    assert np.isclose(Me[0].sum(), vol)
    # stiffness: symmetric, constants in its kernel, PSD
    assert np.allclose(Ke[0], Ke[0].T, atol=1e-13)
    assert np.allclose(Ke[0].sum(axis=1), 0.0, atol=1e-12)
    assert np.linalg.eigvalsh(Ke[0]).min() > -1e-12
    # K_e reproduces int |grad u|^2 for u = x_0 (= |T|)
    u = xyz[:, 0]
    assert np.isclose(u @ Ke[0] @ u, vol)


@pytest.mark.parametrize("dim", [2, 3])
def test_element_divergence_matrix(dim):
    """D_e[c][A][B] = -int d_c M_A N_B: for u = e_c x_c (div u = 1) the
    pressure-row action sum_A D[c][A][B] u_A = -int N_B = -|T|/(d+1)."""
    xyz, conn, vol = _one_element(dim)
    _, _, De = fem.element_matrices(xyz, conn, dim)
    for c in range(dim):
        got = De[0, c].T @ xyz[:, c]
        assert np.allclose(got, -vol / (dim + 1))
        # sum over B of D[c][A][B] = -int d_c M_A: total over A is zero
        assert abs(De[0, c].sum()) < 1e-14


# --------------------------------------------------------- global system

def test_channel_counts_match_golden():
    """Structured 32x8 channel: node, vertex and pattern counts."""
    g = json.load(open(os.path.join(GOLDEN, "channel_32x8_counts.json")))
    m = meshes.channel2d()
    pat = fem.patterns(m["xyz"].shape[0], m["n_vertices"], m["conn"], 2)
    assert m["xyz"].shape[0] == g["N"] and m["n_vertices"] == g["P"]
    assert pat["S"][1].size == g["nnz_S"] and pat["G"][1].size == g["nnz_G"]
    assert pat["GT"][1].size == g["nnz_G"]
    assert 2 * m["xyz"].shape[0] + m["n_vertices"] == g["n_dof"]


def _brute_pattern(conn, ncols_filter=None):
    rows = {}
    for el in conn:
        for a in el:
            s = rows.setdefault(int(a), set())
            for b in el:
                if ncols_filter is None or b < ncols_filter:
                    s.add(int(b))
    return rows


@pytest.mark.parametrize("kind", ["channel", "pipe"])
def test_pattern_brute_force(kind):
    m = meshes.channel2d(4, 2) if kind == "channel" else meshes.pipe3d(n_c=2, n_r=1, n_x=2)
    N, P = m["xyz"].shape[0], m["n_vertices"]
    pat = fem.patterns(N, P, m["conn"], m["dim"])
    br = _brute_pattern(m["conn"])
    rp, col = pat["S"]
    for r in range(N):
        assert list(col[rp[r]:rp[r + 1]]) == sorted(br.get(r, set()))
    rp, col = pat["G"]
    for r in range(N):
        assert list(col[rp[r]:rp[r + 1]]) == sorted(b for b in br.get(r, set()) if b < P)
    rp, col = pat["GT"]
    for r in range(P):
        assert list(col[rp[r]:rp[r + 1]]) == sorted(br.get(r, set()))


@pytest.mark.parametrize("kind", ["channel", "pipe"])
def test_global_matrix_invariants(kind):
    m = meshes.channel2d(8, 4) if kind == "channel" else meshes.pipe3d(n_c=2, n_r=2, n_x=4, length=2.0)
    mats = fem.assemble(m)
    Ms, Ks = mats["Ms"], mats["Ks"]
    # exact pattern (structural zeros kept)
    pat = fem.patterns(mats["N"], mats["P"], m["conn"], m["dim"])
    assert np.array_equal(Ms.indptr, pat["S"][0]) and np.array_equal(Ms.indices, pat["S"][1])
    assert np.array_equal(mats["D"][0].indptr, pat["G"][0]) and np.array_equal(mats["D"][0].indices, pat["G"][1])
    assert abs(Ms - Ms.T).max() < 1e-15 * abs(Ms).max() * 10
    assert abs(Ks - Ks.T).max() < 1e-13 * abs(Ks).max()
    # 1^T M 1 = |Omega| (discrete volume), K 1 = 0
    vol = 4.0 if kind == "channel" else None
    one = np.ones(mats["N"])
    if vol is not None:
        assert np.isclose(one @ Ms @ one, vol, rtol=1e-13)
    assert np.abs(Ks @ one).max() < 1e-11 * abs(Ks).max()
    # M positive definite (Cholesky of the dense matrix)
    np.linalg.cholesky(Ms.toarray())
    # D^T applied to the nodal interpolant of u = (x, 0[, 0]) is -int N_B
    u = np.zeros((mats["N"], m["dim"]))
    u[:, 0] = m["xyz"][:, 0]
    dtu = mats["D"][0].T @ u[:, 0]
    Mp, _ = fem.p1_diagonals(m)
    P = mats["P"]
    assert np.isclose(dtu.sum(), -(one @ Ms @ one), rtol=1e-12)


def test_p1_diagonals_closed_form():
    """diag of the P1 mass: int lambda_a^2 = 2|T|/((d+1)(d+2)); summed over the
    vertices this is 2|Omega|/(d+2)."""
    for m in (meshes.channel2d(6, 3), meshes.pipe3d(n_c=2, n_r=1, n_x=3, length=1.5)):
        mats = fem.assemble(m)
        d = m["dim"]
        Mp, Lp = fem.p1_diagonals(m)
        vol = np.ones(mats["N"]) @ mats["Ms"] @ np.ones(mats["N"])
        assert np.isclose(Mp.sum(), 2 * vol / (d + 2), rtol=1e-12)
        assert np.all(Lp > 0)


def test_saddle_matrix_complex_symmetric():
    wl = workloads.channel_workload(8, 4, n_modes=3)
    mats = fem.assemble(wl["mesh"])
    A = fem.saddle_matrix(mats, wl["omegas"][2], 1.0, 0.01)
    rng = np.random.default_rng(3)
    n = A.shape[0]
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    y = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    assert abs(x @ (A @ y) - y @ (A @ x)) < 1e-12 * abs(x @ (A @ y))
    assert abs(A - A.T).max() < 1e-14 * abs(A).max()
    # not Hermitian for omega > 0
    assert abs(A - A.conj().T).max() > 0


# -------------------------------------------------------------- solutions

def test_channel_mode0_recovers_poiseuille_exactly():
    """The steady parabola and the linear pressure lie in P2 x P1, so the
    discrete solution equals the analytic one up to rounding (Sec. 3.2)."""
    wl = workloads.channel_workload(n_modes=1)
    mats = fem.assemble(wl["mesh"])
    X = fem.solve_modes(mats, wl)
    u, p = fem.split_fields(mats, X[0])
    ue, pe = workloads.exact_nodal(wl, 0)
    assert fem.relative_l2_error(mats["Ms"], ue, u) < 1e-12
    assert np.abs(p - pe).max() < 1e-10 * np.abs(pe).max()
    assert np.abs(X[0].imag).max() == 0.0


def test_channel_third_order_convergence():
    """e proportional to h^3 at a resolved mode (Eq. int_error, Sec. 3.4)."""
    errs = []
    for s in (1, 2):
        wl = workloads.channel_workload(16 * s, 4 * s, n_modes=2)
        mats = fem.assemble(wl["mesh"])
        X = fem.solve_modes(mats, wl)
        u, _ = fem.split_fields(mats, X[1])
        ue, _ = workloads.exact_nodal(wl, 1)
        errs.append(fem.relative_l2_error(mats["Ms"], ue, u))
    assert errs[0] / errs[1] > 6.0


def test_solution_linear_in_boundary_data():
    wl = workloads.channel_workload(8, 4, n_modes=3)
    mats = fem.assemble(wl["mesh"])
    X1 = fem.solve_modes(mats, wl)
    wl2 = dict(wl)
    wl2["g"] = wl["g"] * (2.0 - 3.0j)
    X2 = fem.solve_modes(mats, wl2)
    assert np.abs(X2 - (2.0 - 3.0j) * X1).max() < 1e-11 * np.abs(X2).max()


def test_discrete_divergence_vanishes():
    """Continuity rows: D^T u (including the Dirichlet part) = 0."""
    wl = workloads.channel_workload(8, 4, n_modes=3)
    mats = fem.assemble(wl["mesh"])
    X = fem.solve_modes(mats, wl)
    d, N = 2, mats["N"]
    for k in range(3):
        u = X[k, : d * N].reshape(N, d)
        div = sum(mats["D"][c].T @ u[:, c] for c in range(d))
        assert np.abs(div).max() < 1e-11 * np.abs(u).max()
    assert np.all(fem.relative_residual(mats, wl, X) < 1e-12)


def test_tiny_mesh_sparse_lu_matches_dense_solve():
    wl = workloads.channel_workload(2, 1, n_modes=3)
    mats = fem.assemble(wl["mesh"])
    X = fem.solve_modes(mats, wl)
    dd = fem.dirichlet_dofs(wl["dir_nodes"], 2)
    for k in range(3):
        A = fem.saddle_matrix(mats, wl["omegas"][k], wl["rho"], wl["mu"])
        A_FF, b_F, free = fem.lifted_system(A, dd, wl["g"][k].reshape(-1))
        xd = np.linalg.solve(A_FF.toarray(), b_F)
        assert np.abs(xd - X[k, free]).max() < 1e-12 * max(1.0, np.abs(xd).max())


def test_masked_apply_consistent_with_rhs_and_solution():
    """A_hat x = b for the exact solution (identity Dirichlet rows)."""
    wl = workloads.channel_workload(8, 4, n_modes=3)
    mats = fem.assemble(wl["mesh"])
    X = fem.solve_modes(mats, wl)
    B = fem.rhs_block(mats, wl)
    Y = fem.masked_apply(mats, wl["omegas"], wl["rho"], wl["mu"], wl["dir_nodes"], X.T.copy())
    assert np.abs(Y - B).max() < 1e-10 * np.abs(B).max()


def test_small_pipe_close_to_womersley():
    """Polygonal straight-sided pipe: mode errors against the J0 profile are
    small and shrink with refinement (Sec. 3.4)."""
    errs = []
    for n_c, n_r, n_x in ((2, 1, 4), (4, 2, 8)):
        wl = workloads.pipe_workload(n_c=n_c, n_r=n_r, n_x=n_x, n_modes=2, length=2.0, jitter=0.0)
        mats = fem.assemble(wl["mesh"])
        X = fem.solve_modes(mats, wl)
        u, _ = fem.split_fields(mats, X[1])
        ue, _ = workloads.exact_nodal(wl, 1)
        errs.append(fem.relative_l2_error(mats["Ms"], ue, u))
    assert errs[1] < errs[0] and errs[1] < 0.05


# ----------------------------------------------------------- reconstruction

def test_reconstruction_single_mode_and_parseval():
    rng = np.random.default_rng(5)
    n_t, T = 16, 2.0
    om = 2 * np.pi * np.arange(4) / T
    U = rng.standard_normal((4, 7)) + 1j * rng.standard_normal((4, 7))
    U[0] = U[0].real
    ut = fem.reconstruct(U, om, n_t, T)
    t = np.arange(n_t) * T / n_t
    one = fem.reconstruct(U[2:3], om[2:3], n_t, T)
    assert np.allclose(one, (U[2][None, :] * np.exp(1j * om[2] * t)[:, None]).real)
    # mean over a period of u^2 = u_0^2 + 1/2 sum_k |u_k|^2 (k >= 1, k < n_t/2)
    lhs = (ut ** 2).mean(axis=0)
    rhs = U[0].real ** 2 + 0.5 * (np.abs(U[1:]) ** 2).sum(axis=0)
    assert np.allclose(lhs, rhs)


# ---------------------------------------------------------- analytic inputs

def test_womersley_profiles_solve_their_odes():
    """j w rho u = G + mu u'' (channel), + mu (u'' + u'/r) (pipe), u = 0 on the wall."""
    rho, mu, G = 1.0, 0.01, 1.0
    H, w = 0.5, 2 * np.pi * 3
    y = np.linspace(-0.45, 0.45, 7)
    h = 1e-4
    u = lambda s: channel_profile(s, w, H, rho, mu, G)
    upp = (u(y + h) - 2 * u(y) + u(y - h)) / h ** 2
    assert np.allclose(1j * w * rho * u(y), G + mu * upp, rtol=1e-5, atol=1e-6)
    assert abs(u(np.array([H]))[0]) < 1e-12 and abs(u(np.array([-H]))[0]) < 1e-12
    R, mu2 = 1.0, 0.2
    r = np.linspace(0.1, 0.9, 7)
    v = lambda s: pipe_profile(s, w, R, rho, mu2, G)
    vpp = (v(r + h) - 2 * v(r) + v(r - h)) / h ** 2
    vp = (v(r + h) - v(r - h)) / (2 * h)
    assert np.allclose(1j * w * rho * v(r), G + mu2 * (vpp + vp / r), rtol=1e-5, atol=1e-6)
    assert abs(v(np.array([R]))[0]) < 1e-12
    # small omega tends to the steady parabola
    assert np.allclose(channel_profile(y, 1e-7, H, rho, mu, G), channel_profile(y, 0.0, H, rho, mu, G), rtol=1e-5)
    assert np.allclose(pipe_profile(r, 1e-7, R, rho, mu2, G), pipe_profile(r, 0.0, R, rho, mu2, G), rtol=1e-5)


def test_pipe_generator_is_conforming():
    """Every interior face of the generated tet mesh is shared by exactly two
    tets and every boundary face lies on the wall, inlet or outlet."""
    m = meshes.pipe3d(n_c=3, n_r=2, n_x=3, length=2.0)
    tets = m["conn"][:, :4]
    faces = {}
    for t in tets:
        for f in ((0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)):
            key = tuple(sorted(int(t[i]) for i in f))
            faces[key] = faces.get(key, 0) + 1
    assert max(faces.values()) == 2
    tag = m["tag"]
    for f, cnt in faces.items():
        if cnt == 1:
            common = tag[f[0]] & tag[f[1]] & tag[f[2]]
            assert common != 0


def test_bifurcation_generator_is_conforming_and_tagged():
    """Voxel bifurcation: every interior face is shared by exactly two tets;
    the nodes of every boundary triangle (vertices and edge nodes) carry a
    common tag, interior nodes carry none; inlet, outlet and wall all exist
    and some outlet nodes are not wall nodes (a natural outflow boundary)."""
    m = meshes.bifurcation3d(h=0.4)
    conn = m["conn"]
    tets = conn[:, :4].astype(np.int64)
    P = m["n_vertices"]
    local = ((0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3))
    f = np.sort(np.concatenate([tets[:, list(t)] for t in local], axis=0), axis=1)
    keys = (f[:, 0] * P + f[:, 1]) * P + f[:, 2]
    uk, idx, cnt = np.unique(keys, return_index=True, return_counts=True)
    assert cnt.max() == 2
    tag = m["tag"]
    bf = f[idx[cnt == 1]]
    assert np.all((tag[bf[:, 0]] & tag[bf[:, 1]] & tag[bf[:, 2]]) != 0)
    # boundary nodes: vertices of boundary faces and the edge nodes of their edges
    on_b = np.zeros(tag.size, dtype=bool)
    on_b[bf.ravel()] = True
    edges = {(min(int(a), int(b)), max(int(a), int(b))) for tri in bf for a, b in ((tri[0], tri[1]), (tri[1], tri[2]),
                                                                                      (tri[0], tri[2]))}
    pairs = ((0, 1), (1, 2), (2, 0), (0, 3), (1, 3), (2, 3))
    for e in range(conn.shape[0]):
        for j, (a, b) in enumerate(pairs):
            u, w = int(conn[e, a]), int(conn[e, b])
            if (min(u, w), max(u, w)) in edges:
                on_b[conn[e, 4 + j]] = True
    assert np.array_equal(on_b, tag != 0)
    assert (tag & meshes.INLET).any() and (tag & meshes.WALL).any()
    assert ((tag & meshes.OUTLET) != 0).sum() > 0 and (((tag & meshes.OUTLET) != 0) & ((tag & meshes.WALL) == 0)).any()


# -------------------------------------------------- L2 norm and P1 mass

def test_l2_norm_closed_forms_on_the_channel():
    """On [0,4] x [-0.5,0.5]: ||1|| = 2, ||x||^2 = 64/3, ||x^2||^2 = 4^5/5,
    ||(1, y)||^2 = 4 + 1/3 (P2 reproduces polynomials of degree 2 exactly and
    M_s integrates their products exactly); relative errors scale linearly."""
    m = meshes.channel2d(8, 4)
    mats = fem.assemble(m)
    x, y = m["xyz"][:, 0], m["xyz"][:, 1]
    one = np.ones_like(x)
    assert abs(fem.l2_norm(mats["Ms"], one) - 2.0) < 1e-13
    assert abs(fem.l2_norm(mats["Ms"], x) - math.sqrt(64.0 / 3.0)) < 1e-12
    assert abs(fem.l2_norm(mats["Ms"], x * x) - math.sqrt(4.0 ** 5 / 5.0)) < 1e-11
    assert abs(fem.l2_norm(mats["Ms"], np.stack([one, y], axis=1)) - math.sqrt(4.0 + 1.0 / 3.0)) < 1e-12
    assert abs(fem.relative_l2_error(mats["Ms"], x, 0.75 * x) - 0.25) < 1e-14
    # complex fields: ||(1 + 2j) x|| = sqrt(5) ||x||
    assert abs(fem.l2_norm(mats["Ms"], (1 + 2j) * x) - math.sqrt(5.0 * 64.0 / 3.0)) < 1e-11


def test_p1_mass_closed_forms():
    """Full P1 mass matrix: 1^T M 1 = |Omega|, x^T M 1 = int x, x^T M x = int x^2
    (the P1 interpolant of a linear function is exact), symmetric, and the
    element matrix |T|/12 [2 1 1; 1 2 1; 1 1 2] on a single triangle."""
    m = meshes.channel2d(8, 4)
    Mp = fem.p1_mass(m).toarray()
    P = m["n_vertices"]
    x = m["xyz"][:P, 0]
    one = np.ones(P)
    assert np.allclose(Mp, Mp.T, atol=0)
    assert abs(one @ Mp @ one - 4.0) < 1e-13
    assert abs(x @ Mp @ one - 8.0) < 1e-12
    assert abs(x @ Mp @ x - 64.0 / 3.0) < 1e-12
    tri = dict(xyz=np.array([[0.0, 0.0], [2.0, 0.0], [0.0, 1.0], [1.0, 0.0], [1.0, 0.5], [0.0, 0.5]]),
               conn=np.array([[0, 1, 2, 3, 4, 5]], dtype=np.int32), dim=2, n_vertices=3)
    ref = (1.0 / 12.0) * np.array([[2, 1, 1], [1, 2, 1], [1, 1, 2]])
    assert np.allclose(fem.p1_mass(tri).toarray(), ref, atol=1e-15)
    # 3D: 1^T M 1 is the discrete volume
    pm = meshes.pipe3d(n_c=2, n_r=1, n_x=3, length=1.0, jitter=0.0)
    M3 = fem.p1_mass(pm)
    vol = fem.assemble(pm)["Ms"].sum()
    assert abs(M3.sum() - vol) < 1e-12 * vol
    Wu, Wp = fem.block_weights(fem.assemble(m), m)
    assert Wu.shape == (2 * m["xyz"].shape[0],) * 2 and Wp.shape == (P, P)


def test_p1_stiffness_closed_forms():
    """Full P1 stiffness matrix: K 1 = 0 (constants have no gradient), the energy of
    a linear function is int |grad u|^2 = |a|^2 |Omega| (x^T K x = 4 and
    (x + 2y)^T K (x + 2y) = 20 on the 4 x 1 channel), symmetric positive
    semidefinite, its diagonal is the one p1_diagonals gives, and on one
    right triangle with legs 2 and 1 it is the textbook element matrix."""
    m = meshes.channel2d(8, 4)
    K = fem.p1_stiffness(m).toarray()
    P = m["n_vertices"]
    x, y = m["xyz"][:P, 0], m["xyz"][:P, 1]
    assert np.allclose(K, K.T, atol=0)
    assert np.abs(K @ np.ones(P)).max() < 1e-12
    assert abs(x @ K @ x - 4.0) < 1e-12
    assert abs((x + 2 * y) @ K @ (x + 2 * y) - 20.0) < 1e-11
    assert np.linalg.eigvalsh(K).min() > -1e-12
    _, Ld = fem.p1_diagonals(m)
    assert np.allclose(np.diag(K), Ld, rtol=1e-13)
    tri = dict(xyz=np.array([[0.0, 0.0], [2.0, 0.0], [0.0, 1.0], [1.0, 0.0], [1.0, 0.5], [0.0, 0.5]]),
               conn=np.array([[0, 1, 2, 3, 4, 5]], dtype=np.int32), dim=2, n_vertices=3)
    # grad l_1 = (1/2, 0), grad l_2 = (0, 1), grad l_0 = (-1/2, -1); area 1
    g = np.array([[-0.5, -1.0], [0.5, 0.0], [0.0, 1.0]])
    assert np.allclose(fem.p1_stiffness(tri).toarray(), g @ g.T, atol=1e-15)
    # 3D pipe: K 1 = 0 and x^T K x = |Omega| (the discrete volume)
    pm = meshes.pipe3d(n_c=2, n_r=1, n_x=3, length=1.0, jitter=0.0)
    K3 = fem.p1_stiffness(pm)
    x3 = pm["xyz"][:pm["n_vertices"], 0]
    vol = fem.assemble(pm)["Ms"].sum()
    assert np.abs(K3 @ np.ones(pm["n_vertices"])).max() < 1e-12
    assert abs(x3 @ K3 @ x3 - vol) < 1e-12 * vol
