"""Pins of the oracle's isoparametric (curved) P2 elements (no GPU).

The paper projects inserted boundary nodes onto curved walls (Sec. 3.1);
elements whose edge nodes are displaced are integrated with the quadratic
geometry map.  Pins: straight elements give the exact affine matrices; the
area of a triangle with one parabolic edge has a closed form; constants have
zero stiffness; the divergence of the coordinate field is the element area;
the isoparametric area of an annulus converges at fourth order where the
straight-sided one is second order; and the Stokes flow in a curved channel
(an exact solution, r ln r profile) converges at third order on curved
elements.""" 
import math

import numpy as np
import pytest

from oracle import boundary, fem
from synthetic import meshes


def _tri(delta):
    xyz = np.array([[0.0, 0.0], [2.0, 0.0], [0.0, 1.0], [1.0, -delta], [1.0, 0.5], [0.0, 0.5]])
    return xyz, np.array([[0, 1, 2, 3, 4, 5]], dtype=np.int64)


def test_iso_equals_affine_on_straight_elements():
    m = meshes.pipe3d(n_c=2, n_r=1, n_x=2, length=1.0, jitter=0.05)
    conn = m["conn"].astype(np.int64)
    assert not fem.curved_elements(m["xyz"], conn, 3).any()
    a = fem.element_matrices(m["xyz"], conn, 3)
    b = fem.element_matrices_iso(m["xyz"], conn, 3)
    for x, y in zip(a, b):
        assert np.abs(x - y).max() < 1e-13 * np.abs(x).max()


@pytest.mark.parametrize("delta", [0.05, 0.2])
def test_parabolic_edge_triangle_closed_forms(delta):
    """Area = |T| + (2/3) |chord| delta for the edge node displaced by delta
    (the quadratic edge bulges by 4 delta t (1 - t)); K 1 = 0; the discrete
    divergence of the coordinate field x gives minus the area."""
    xyz, conn = _tri(delta)
    assert fem.curved_elements(xyz, conn, 2).all()
    Me, Ke, De = fem.element_matrices_iso(xyz, conn, 2)
    area = 1.0 + (2.0 / 3.0) * 2.0 * delta
    assert abs(Me[0].sum() - area) < 1e-14
    assert np.abs(Ke[0].sum(axis=1)).max() < 1e-13
    assert np.allclose(Me[0], Me[0].T, atol=1e-15) and np.allclose(Ke[0], Ke[0].T, atol=1e-13)
    # sum_a x_a D_x[a][b] = -int d_x(x) psi_b = -int psi_b; summed over b: -area
    assert abs(xyz[:, 0] @ De[0, 0] @ np.ones(3) + area) < 1e-13
    assert abs(xyz[:, 1] @ De[0, 1] @ np.ones(3) + area) < 1e-13
    # the first moment int x = sum_ab x_a M_ab: exact by quadrature of a polynomial
    pts, w = fem.simplex_rule(2, 8)
    phi, dphi = fem.p2_basis(2, pts)
    J = np.einsum("ar,qai->qri", xyz, dphi)
    ref = float(np.sum(w * np.linalg.det(J) * (phi @ xyz[:, 0])))
    assert abs(xyz[:, 0] @ Me[0] @ np.ones(6) - ref) < 1e-13


def test_annulus_area_converges_at_fourth_order():
    exact = 0.25 * math.pi * (2.0 ** 2 - 1.0 ** 2)
    e_iso, e_str = [], []
    for n in (4, 8, 16):
        for curved, out in ((True, e_iso), (False, e_str)):
            m = meshes.annulus2d(n_r=n // 2, n_t=2 * n, curved=curved)
            out.append(abs(fem.assemble(m)["Ms"].sum() - exact))
    assert e_iso[0] / e_iso[1] > 12 and e_iso[1] / e_iso[2] > 12, e_iso
    assert 3 < e_str[0] / e_str[1] < 5, e_str


def _curved_channel(n_r, n_t, curved, mu=1.0, K=1.0, r1=1.0, r2=2.0, theta=0.5 * np.pi):
    """Steady Stokes flow in the annular sector driven by p = K (theta_max - t):
    u = u_t(r) e_t, u_t = A r + B / r - K / (2 mu) r ln r with u_t(r1) = u_t(r2) = 0;
    Dirichlet inlet (t = 0) and walls, the exact pseudo-traction
    (-p I + mu grad u) n = -mu u_t / r e_r at the outlet (t = theta_max)."""
    m = meshes.annulus2d(n_r=n_r, n_t=n_t, r1=r1, r2=r2, theta=theta, curved=curved)
    c = K / (2.0 * mu)
    A = c * (r2 * math.log(r2) - r1 * r1 / r2 * math.log(r1)) / (r2 - r1 * r1 / r2)
    B = c * r1 * r1 * math.log(r1) - A * r1 * r1
    ut = lambda r: A * r + B / r - c * r * np.log(r)
    xyz = m["xyz"]
    r = np.hypot(xyz[:, 0], xyz[:, 1])
    t = np.arctan2(xyz[:, 1], xyz[:, 0])
    uex = np.stack([-np.sin(t) * ut(r), np.cos(t) * ut(r)], axis=1)
    tag = m["tag"]
    dn = np.flatnonzero((tag & (meshes.WALL | meshes.INLET)) != 0)
    g = uex[dn][None].astype(np.complex128)
    h = np.zeros_like(xyz)
    h[:, 0] = -mu * ut(r) / r * math.cos(theta)
    h[:, 1] = -mu * ut(r) / r * math.sin(theta)
    faces = boundary.boundary_faces(m, meshes.OUTLET)
    load = boundary.neumann_load(m, faces, h)[None].astype(np.complex128)
    wl = dict(mesh=m, omegas=np.array([0.0]), rho=1.0, mu=mu, dir_nodes=dn, g=g, load=load)
    mats = fem.assemble(m)
    X = fem.solve_modes(mats, wl)
    u, _ = fem.split_fields(mats, X[0])
    return fem.relative_l2_error(mats["Ms"], uex, u)


def test_curved_channel_converges_at_third_order():
    """The exact curved-channel flow is reproduced at (at least) third order on
    isoparametric elements (measured ratios 10.8, 12.3, 12.6 per halving)."""
    e = [_curved_channel(n, 4 * n, True) for n in (2, 4, 8)]
    assert e[0] < 1e-2 and e[0] / e[1] > 8.0 and e[1] / e[2] > 8.0, e
