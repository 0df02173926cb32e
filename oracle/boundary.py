"""FP64 CPU oracle of the Neumann (traction) boundary term (test
infrastructure: only the tests, ``__graft_entry__.smoke`` and the CPU-baseline
leg of ``bench.py`` use it; it imports nothing from the product).

What it computes (arXiv 2009.06725, Sec. 2.3): the boundary integral of the
weak form, b_u[A, c] = int_{Gamma_h} M_A h_c dGamma (Eq. LS_construction), for a
traction h given by its nodal values and interpolated with the P2 trace
basis, i.e. b_u = M_Gamma h with M_Gamma the boundary mass matrix of the P2
faces on Gamma_h (segments with 3 nodes in 2D, triangles with 6 nodes in 3D).
Gamma_h is the set of element faces whose nodes all carry a given tag bit and
that belong to one element only.  Straight faces: |F| / |F_ref| times the
reference matrix; curved faces (an edge node off its edge midpoint, the
paper's projected boundary nodes, Sec. 3.1): the isoparametric face map
x(xi) = sum_a x_a phi_a(xi) and its surface Jacobian at every point of a
6-point-per-direction Gauss rule.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as spm

# local P2 faces of an element, each in the face's own VTK order
# (vertices a, b[, c], then the edge nodes (a,b)[, (b,c), (c,a)])
FACES_2D = ((0, 1, 3), (1, 2, 4), (2, 0, 5))
FACES_3D = ((0, 1, 2, 4, 5, 6), (0, 1, 3, 4, 8, 7), (1, 2, 3, 5, 9, 8), (2, 0, 3, 6, 7, 9))


def _p2_trace_basis(fdim, pts):
    """P2 basis on the reference face (segment [0,1] or unit triangle) in barycentrics:
    vertex functions lam (2 lam - 1), edge functions 4 lam_a lam_b."""
    lam = np.concatenate([1.0 - pts.sum(axis=1, keepdims=True), pts], axis=1)
    vals = [lam[:, a] * (2 * lam[:, a] - 1) for a in range(fdim + 1)]
    edges = ((0, 1),) if fdim == 1 else ((0, 1), (1, 2), (2, 0))
    vals += [4 * lam[:, a] * lam[:, b] for a, b in edges]
    return np.stack(vals, axis=1)


def _face_rule(fdim, n=4):
    g, wg = np.polynomial.legendre.leggauss(n)
    g, wg = 0.5 * (g + 1.0), 0.5 * wg
    if fdim == 1:
        return g[:, None], wg
    u, v = np.meshgrid(g, g, indexing="ij")
    wu, wv = np.meshgrid(wg, wg, indexing="ij")
    return np.stack([u.ravel(), (v * (1 - u)).ravel()], axis=1), (wu * wv * (1 - u)).ravel()


def _p2_trace_grads(fdim, pts):
    """Reference derivatives [Q][nl][fdim] of the P2 trace basis."""
    lam = np.concatenate([1.0 - pts.sum(axis=1, keepdims=True), pts], axis=1)
    dlam = np.zeros((fdim + 1, fdim))
    dlam[0, :] = -1.0
    dlam[1:, :] = np.eye(fdim)
    g = [(4 * lam[:, a] - 1)[:, None] * dlam[a][None, :] for a in range(fdim + 1)]
    edges = ((0, 1),) if fdim == 1 else ((0, 1), (1, 2), (2, 0))
    g += [4 * (lam[:, a][:, None] * dlam[b][None, :] + lam[:, b][:, None] * dlam[a][None, :]) for a, b in edges]
    return np.stack(g, axis=1)


def curved_faces(mesh, faces, rtol=1e-12):
    """Faces whose edge nodes are not at their edge midpoints."""
    xyz = mesh["xyz"]
    fdim = mesh["dim"] - 1
    edges = ((0, 1),) if fdim == 1 else ((0, 1), (1, 2), (2, 0))
    out = np.zeros(faces.shape[0], dtype=bool)
    for j, (a, b) in enumerate(edges):
        xa, xb, xm = xyz[faces[:, a]], xyz[faces[:, b]], xyz[faces[:, fdim + 1 + j]]
        out |= np.linalg.norm(xm - 0.5 * (xa + xb), axis=1) > rtol * np.linalg.norm(xb - xa, axis=1)
    return out


def face_mass_iso(mesh, faces, n=6):
    """Face mass matrices [n_f][nl][nl] of the isoparametric P2 faces:
    sum_q w_q J_s(xi_q) phi_a phi_b with J_s = |dx/dxi| (segment) or
    |dx/dxi_1 x dx/dxi_2| (triangle)."""
    fdim = mesh["dim"] - 1
    pts, w = _face_rule(fdim, n)
    phi = _p2_trace_basis(fdim, pts)
    dphi = _p2_trace_grads(fdim, pts)
    X = mesh["xyz"][faces]                            # [F][nl][d]
    T = np.einsum("far,qai->fqir", X, dphi)           # tangents [F][Q][fdim][d]
    if fdim == 1:
        Js = np.linalg.norm(T[:, :, 0, :], axis=2)
    else:
        Js = np.linalg.norm(np.cross(T[:, :, 0, :], T[:, :, 1, :]), axis=2)
    return np.einsum("fq,q,qa,qb->fab", Js, w, phi, phi)


def face_mass_reference(fdim):
    """int phi_a phi_b over the reference face (length 1 or area 1/2)."""
    pts, w = _face_rule(fdim)
    phi = _p2_trace_basis(fdim, pts)
    return np.einsum("q,qa,qb->ab", w, phi, phi)


def boundary_faces(mesh, bit):
    """P2 faces [n_f][3 or 6] (node ids, face VTK order) of Gamma_h: faces of one element
    only whose nodes all carry tag bit."""
    conn, tag, dim = mesh["conn"].astype(np.int64), mesh["tag"], mesh["dim"]
    local = FACES_2D if dim == 2 else FACES_3D
    nv = dim  # vertices per face
    count = {}
    cand = []
    for e in range(conn.shape[0]):
        for f in local:
            nodes = conn[e, list(f)]
            key = tuple(sorted(nodes[:nv].tolist()))
            count[key] = count.get(key, 0) + 1
            if np.all((tag[nodes] & bit) != 0):
                cand.append((key, nodes))
    return np.array([nodes for key, nodes in cand if count[key] == 1], dtype=np.int64).reshape(-1, 3 if dim == 2 else 6)


def face_measures(mesh, faces):
    xyz = mesh["xyz"]
    if mesh["dim"] == 2:
        return np.linalg.norm(xyz[faces[:, 1]] - xyz[faces[:, 0]], axis=1)
    a, b, c = xyz[faces[:, 0]], xyz[faces[:, 1]], xyz[faces[:, 2]]
    return 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)


def face_mass(mesh, faces):
    """Boundary mass matrix M_Gamma (N x N, sparse) of the P2 faces."""
    N = mesh["xyz"].shape[0]
    fdim = mesh["dim"] - 1
    Mref = face_mass_reference(fdim)
    ref_measure = 1.0 if fdim == 1 else 0.5
    meas = face_measures(mesh, faces)
    nl = faces.shape[1]
    rows = np.repeat(faces, nl, axis=1).ravel()
    cols = np.tile(faces, (1, nl)).ravel()
    Mf = meas[:, None, None] / ref_measure * Mref[None]
    cv = curved_faces(mesh, faces)
    if cv.any():
        Mf[cv] = face_mass_iso(mesh, faces[cv])
    vals = Mf.ravel()
    return spm.coo_matrix((vals, (rows, cols)), shape=(N, N)).tocsr()


def neumann_load(mesh, faces, h):
    """b_u [N][d] = M_Gamma h for nodal tractions h [N][d] (complex or real)."""
    Mg = face_mass(mesh, faces)
    h = np.asarray(h)
    return np.stack([Mg @ h[:, c] for c in range(h.shape[1])], axis=1)
