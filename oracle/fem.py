"""FP64 CPU oracle of the per-mode complex Stokes solve (test infrastructure).

This module is the plain definition the CUDA path is checked against.  It is
used only by the tests, by ``__graft_entry__.smoke`` and by the CPU-baseline
leg of ``bench.py``; the product path never imports it, and it imports
nothing from the product.

What it computes (arXiv 2009.06725):
  * P2 velocity / P1 pressure Taylor-Hood simplices (Sec. 2.3),
  * mode-independent real matrices M_s = int M_A M_B, K_s = int grad M_A .
    grad M_B, D_c = -int d_c M_A N_B (Eq. LS_construction, with the
    viscous term mu grad u of Eq. weak_stokes, so the vector operator is
    I_d (x) K_s),
  * the saddle-point matrix A(omega) = [I_d (x) (mu K_s + j omega rho M_s), D; D^T, 0]
    (Eq. linear_sys_def; continuity row multiplied by -1 so A is complex
    symmetric),
  * Dirichlet lifting (Eq. shape_fun / dir_dis): velocity dofs of Dirichlet nodes
    are prescribed, their columns moved to the right-hand side of both the
    momentum rows and the continuity rows; an optional Neumann load (the
    boundary integral of Eq. LS_construction, oracle/boundary.py) is added to
    the momentum rows,
  * an exact sparse direct solve per mode (SuperLU, complex128),
  * reconstruction in time (Eq. sol_reconstruct) and the relative L2 error
    (Eq. total_error) with the L2(Omega) norm evaluated with M_s.
Element integrals use a collapsed (Duffy) Gauss-Legendre rule on the
reference simplex, exact for the polynomial degrees involved.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as spm
import scipy.sparse.linalg as sla

# ---------------------------------------------------------------- quadrature


def simplex_rule(dim, n=5):
    """Collapsed Gauss-Legendre rule on the unit reference simplex.

    Triangle: xi = u, eta = v (1-u), Jacobian (1-u).
    Tet: xi = u, eta = v (1-u), zeta = w (1-u)(1-v), Jacobian (1-u)^2 (1-v).
    With n points per direction it integrates every polynomial of degree
    <= 2n - 1 - (dim - 1) exactly (degree 7 for dim=3, n=5)."""
    g, wg = np.polynomial.legendre.leggauss(n)
    g = 0.5 * (g + 1.0)
    wg = 0.5 * wg
    if dim == 2:
        u, v = np.meshgrid(g, g, indexing="ij")
        wu, wv = np.meshgrid(wg, wg, indexing="ij")
        pts = np.stack([u.ravel(), (v * (1 - u)).ravel()], axis=1)
        w = (wu * wv * (1 - u)).ravel()
    elif dim == 3:
        u, v, t = np.meshgrid(g, g, g, indexing="ij")
        wu, wv, wt = np.meshgrid(wg, wg, wg, indexing="ij")
        pts = np.stack([u.ravel(), (v * (1 - u)).ravel(), (t * (1 - u) * (1 - v)).ravel()], axis=1)
        w = (wu * wv * wt * (1 - u) ** 2 * (1 - v)).ravel()
    else:
        raise ValueError("dim must be 2 or 3")
    return pts, w


# ------------------------------------------------------------ P2 / P1 basis

def _edges(dim):
    return ((0, 1), (1, 2), (2, 0)) if dim == 2 else ((0, 1), (1, 2), (2, 0), (0, 3), (1, 3), (2, 3))


def p2_basis(dim, pts):
    """Quadratic Lagrange basis on the reference simplex (Sec. 2.3), VTK order.

    In barycentrics lam_0 = 1 - sum xi, lam_i = xi_i: vertex functions
    lam_a (2 lam_a - 1), edge functions 4 lam_a lam_b.  Returns values
    [Q][nl] and reference gradients [Q][nl][dim]."""
    Q = pts.shape[0]
    lam = np.concatenate([1.0 - pts.sum(axis=1, keepdims=True), pts], axis=1)  # [Q][dim+1]
    dlam = np.zeros((dim + 1, dim))
    dlam[0, :] = -1.0
    dlam[1:, :] = np.eye(dim)
    vals, grads = [], []
    for a in range(dim + 1):
        vals.append(lam[:, a] * (2 * lam[:, a] - 1))
        grads.append((4 * lam[:, a] - 1)[:, None] * dlam[a][None, :])
    for a, b in _edges(dim):
        vals.append(4 * lam[:, a] * lam[:, b])
        grads.append(4 * (lam[:, a][:, None] * dlam[b][None, :] + lam[:, b][:, None] * dlam[a][None, :]))
    return np.stack(vals, axis=1), np.stack(grads, axis=1)


def p1_basis(dim, pts):
    """Linear Lagrange basis (the barycentrics) and reference gradients."""
    lam = np.concatenate([1.0 - pts.sum(axis=1, keepdims=True), pts], axis=1)
    dlam = np.zeros((dim + 1, dim))
    dlam[0, :] = -1.0
    dlam[1:, :] = np.eye(dim)
    return lam, np.broadcast_to(dlam, (pts.shape[0], dim + 1, dim))


def reference_integrals(dim, n=5):
    """Reference-simplex integrals of basis products:
    Mref[a,b] = int phi_a phi_b, Kref[i,j,a,b] = int d_i phi_a d_j phi_b,
    Eref[i,a,b] = int d_i phi_a psi_b (phi P2, psi P1)."""
    pts, w = simplex_rule(dim, n)
    phi, dphi = p2_basis(dim, pts)
    psi, _ = p1_basis(dim, pts)
    Mref = np.einsum("q,qa,qb->ab", w, phi, phi)
    Kref = np.einsum("q,qai,qbj->ijab", w, dphi, dphi)
    Eref = np.einsum("q,qai,qb->iab", w, dphi, psi)
    return Mref, Kref, Eref


def p1_reference_integrals(dim, n=5):
    """P1 reference integrals: mass int psi_a psi_b and stiffness pieces."""
    pts, w = simplex_rule(dim, n)
    psi, dpsi = p1_basis(dim, pts)
    M1 = np.einsum("q,qa,qb->ab", w, psi, psi)
    K1 = np.einsum("q,qai,qbj->ijab", w, dpsi, dpsi)
    return M1, K1


# ------------------------------------------------------------------ geometry

def element_maps(xyz, conn, dim):
    """Affine map x = x_0 + J xi of every element: J [E][d][d] (columns are
    vertex differences), det J and J^{-1}.  Rejects non-positive det."""
    x0 = xyz[conn[:, 0]]
    J = np.stack([xyz[conn[:, i + 1]] - x0 for i in range(dim)], axis=-1)
    det = np.linalg.det(J)
    if np.any(det <= 0.0):
        raise ValueError("element with non-positive Jacobian")
    return J, det, np.linalg.inv(J)


def element_matrices(xyz, conn, dim):
    """Element matrices (Eq. LS_construction) of every affine P2 element.

    M_e = |J| Mref,  K_e = |J| sum_ij (J^-1 J^-T)_ij Kref_ij,
    D_e[c] = -|J| sum_i (J^-1)_ic Eref_i  (grad_x = J^-T grad_xi)."""
    Mref, Kref, Eref = reference_integrals(dim)
    _, det, Jinv = element_maps(xyz, conn, dim)
    Me = det[:, None, None] * Mref[None]
    gamma = np.einsum("eic,ejc->eij", Jinv, Jinv) * det[:, None, None]
    Ke = np.einsum("eij,ijab->eab", gamma, Kref)
    De = -np.einsum("e,eic,iab->ecab", det, Jinv, Eref)
    return Me, Ke, De


def curved_elements(xyz, conn, dim, rtol=1e-12):
    """Elements whose edge nodes are not at their edge midpoints (curved,
    isoparametric P2 geometry; the paper projects boundary edge nodes onto
    the curved wall, Sec. 3.1)."""
    nv = dim + 1
    out = np.zeros(conn.shape[0], dtype=bool)
    for j, (a, b) in enumerate(_edges(dim)):
        xa, xb, xm = xyz[conn[:, a]], xyz[conn[:, b]], xyz[conn[:, nv + j]]
        dev = np.linalg.norm(xm - 0.5 * (xa + xb), axis=1)
        out |= dev > rtol * np.linalg.norm(xb - xa, axis=1)
    return out


ISO_QUAD = 6  # points per direction of the collapsed rule on curved elements


def element_matrices_iso(xyz, conn, dim, n=ISO_QUAD):
    """Element matrices of isoparametric P2 elements (x(xi) = sum_a x_a phi_a(xi)):
    at every quadrature point J = sum_a x_a grad_xi phi_a^T, physical gradients
    grad_x phi_a = J^-T grad_xi phi_a, and
    M_e[a,b] = sum_q w_q |J| phi_a phi_b,  K_e[a,b] = sum_q w_q |J| grad_x phi_a . grad_x phi_b,
    D_e[c,a,b] = -sum_q w_q |J| d_c phi_a psi_b  (psi the P1 basis of the reference
    simplex, mapped with the element).  Rejects non-positive |J| at a point."""
    pts, w = simplex_rule(dim, n)
    phi, dphi = p2_basis(dim, pts)            # [Q][nl], [Q][nl][dim]
    psi, _ = p1_basis(dim, pts)               # [Q][nv]
    X = xyz[conn]                             # [E][nl][dim]
    J = np.einsum("ear,qai->eqri", X, dphi)   # [E][Q][dim][dim]: dx_r / dxi_i
    det = np.linalg.det(J)
    if np.any(det <= 0.0):
        raise ValueError("element with non-positive Jacobian at a quadrature point")
    Jinv = np.linalg.inv(J)                   # [E][Q][i][r]
    G = np.einsum("qai,eqic->eqac", dphi, Jinv)  # grad_x phi_a: sum_i dphi/dxi_i (J^-1)_ic
    wd = det * w[None, :]                     # [E][Q]
    Me = np.einsum("eq,qa,qb->eab", wd, phi, phi)
    Ke = np.einsum("eq,eqac,eqbc->eab", wd, G, G)
    De = -np.einsum("eq,eqac,qb->ecab", wd, G, psi)
    return Me, Ke, De


# --------------------------------------------------------------- assembly

def patterns(n_nodes, n_vertices, conn, dim):
    """Structural CSR patterns (row pointers int64, ascending column ids int32)
    of S (P2 x P2: node pairs sharing an element, diagonal included), G (P2
    rows x P1 columns) and G^T.  Structural zeros are part of the pattern."""
    nv = dim + 1
    c = conn.astype(np.int64)
    out = {}
    for name, rc, cc, nr, ncol in (
        ("S", c, c, n_nodes, n_nodes),
        ("G", c, c[:, :nv], n_nodes, n_vertices),
        ("GT", c[:, :nv], c, n_vertices, n_nodes),
    ):
        rows = np.repeat(rc, cc.shape[1], axis=1).ravel()
        cols = np.tile(cc, (1, rc.shape[1])).ravel()
        key = np.unique(rows * ncol + cols)
        r = key // ncol
        rowptr = np.zeros(nr + 1, dtype=np.int64)
        np.add.at(rowptr, r + 1, 1)
        out[name] = (np.cumsum(rowptr), (key % ncol).astype(np.int32))
    return out


def _coo_to_csr(rows, cols, vals, shape):
    A = spm.coo_matrix((vals, (rows, cols)), shape=shape).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return A


def assemble(mesh):
    """Global real matrices: Ms, Ks (N x N), D = [D_x, D_y(, D_z)] (N x P each).

    Sums element contributions over elements (Eq. LS_construction); explicit
    zeros are kept so every matrix has exactly the structural pattern.
    Straight-sided elements use the exact reference integrals; elements with
    displaced edge nodes (curved boundaries, Sec. 3.1) the isoparametric map
    and quadrature (element_matrices_iso)."""
    xyz, conn, dim, P = mesh["xyz"], mesh["conn"].astype(np.int64), mesh["dim"], mesh["n_vertices"]
    N = xyz.shape[0]
    curved = curved_elements(xyz, conn, dim)
    if curved.any():  # isoparametric elements where the geometry is curved
        Me, Ke, De = element_matrices(xyz, conn, dim) if not curved.all() else (None, None, None)
        Mi, Ki, Di = element_matrices_iso(xyz, conn[curved], dim)
        if Me is None:
            Me, Ke, De = Mi, Ki, Di
        else:
            Me[curved], Ke[curved], De[curved] = Mi, Ki, Di
    else:
        Me, Ke, De = element_matrices(xyz, conn, dim)
    nl = conn.shape[1]
    nv = dim + 1
    rows = np.repeat(conn, nl, axis=1).ravel()
    cols = np.tile(conn, (1, nl)).ravel()
    Ms = _coo_to_csr(rows, cols, Me.ravel(), (N, N))
    Ks = _coo_to_csr(rows, cols, Ke.ravel(), (N, N))
    rg = np.repeat(conn, nv, axis=1).ravel()
    cg = np.tile(conn[:, :nv], (1, nl)).ravel()
    D = [_coo_to_csr(rg, cg, De[:, c].ravel(), (N, P)) for c in range(dim)]
    return dict(Ms=Ms, Ks=Ks, D=D, N=N, P=P, dim=dim)


def p1_diagonals(mesh):
    """Diagonals of the P1 (vertex) mass and stiffness matrices, used by the
    block preconditioner's pressure part."""
    xyz, conn, dim, P = mesh["xyz"], mesh["conn"].astype(np.int64), mesh["dim"], mesh["n_vertices"]
    vc = conn[:, :dim + 1]
    M1, K1 = p1_reference_integrals(dim)
    _, det, Jinv = element_maps(xyz, vc, dim)
    gamma = np.einsum("eic,ejc->eij", Jinv, Jinv) * det[:, None, None]
    mdiag = det[:, None] * np.diag(M1)[None, :]
    kdiag = np.einsum("eij,ijaa->ea", gamma, K1)
    Mp = np.zeros(P)
    Lp = np.zeros(P)
    np.add.at(Mp, vc, mdiag)
    np.add.at(Lp, vc, kdiag)
    return Mp, Lp


# ------------------------------------------------------------ the system

def p1_mass(mesh):
    """Full P1 (vertex) mass matrix int N_A N_B over the simplices of the mesh
    (the L2(Omega) inner product of the pressure space, Sec. 2.3), summed
    element by element from the reference integrals."""
    xyz, conn, dim, P = mesh["xyz"], mesh["conn"].astype(np.int64), mesh["dim"], mesh["n_vertices"]
    vc = conn[:, :dim + 1]
    M1, _ = p1_reference_integrals(dim)
    _, det, _ = element_maps(xyz, vc, dim)
    vals = det[:, None, None] * M1[None, :, :]
    nv = dim + 1
    rows = np.repeat(vc, nv, axis=1).ravel()
    cols = np.tile(vc, (1, nv)).ravel()
    return _coo_to_csr(rows, cols, vals.ravel(), (P, P))


def p1_stiffness(mesh):
    """Full P1 (vertex) stiffness matrix int grad N_A . grad N_B over the
    simplices of the mesh: the Laplacian L_p of the Cahouet-Chabard Schur
    approximation (Sec. 2.3), before any boundary condition is imposed."""
    xyz, conn, dim, P = mesh["xyz"], mesh["conn"].astype(np.int64), mesh["dim"], mesh["n_vertices"]
    vc = conn[:, :dim + 1]
    _, K1 = p1_reference_integrals(dim)
    _, det, Jinv = element_maps(xyz, vc, dim)
    gamma = np.einsum("eic,ejc->eij", Jinv, Jinv) * det[:, None, None]
    vals = np.einsum("eij,ijab->eab", gamma, K1)
    nv = dim + 1
    rows = np.repeat(vc, nv, axis=1).ravel()
    cols = np.tile(vc, (1, nv)).ravel()
    return _coo_to_csr(rows, cols, vals.ravel(), (P, P))


def block_weights(mats, mesh):
    """L2(Omega) inner products of the two field blocks of a modal vector in
    the solver's dof order (velocity dof = node * d + c, then the vertices):
    W_u = M_s (x) I_d on the velocity block, W_p = the P1 mass on the pressure
    block."""
    d = mats["dim"]
    Wu = spm.kron(mats["Ms"], spm.identity(d), format="csr")
    return Wu, p1_mass(mesh)


def dof_count(mats):
    return mats["dim"] * mats["N"] + mats["P"]


def saddle_matrix(mats, omega, rho, mu):
    """A(omega) = [I_d (x) (mu K_s + j omega rho M_s), D; D^T, 0] (Eq. linear_sys_def)
    with velocity dofs ordered node-major (dof = node*d + c), then the P
    pressure dofs.  Complex symmetric: A^T = A."""
    d, N, P = mats["dim"], mats["N"], mats["P"]
    Kw = (mu * mats["Ks"] + 1j * omega * rho * mats["Ms"]).tocsr()
    Auu = spm.kron(Kw, spm.identity(d, format="csr"), format="csr")
    # D_full[A*d + c, B] = D_c[A, B]
    blocks = []
    for c in range(d):
        Dc = mats["D"][c].tocoo()
        blocks.append((Dc.row * d + c, Dc.col, Dc.data))
    r = np.concatenate([b[0] for b in blocks])
    cc = np.concatenate([b[1] for b in blocks])
    v = np.concatenate([b[2] for b in blocks])
    Dfull = spm.coo_matrix((v, (r, cc)), shape=(d * N, P)).tocsr()
    A = spm.bmat([[Auu, Dfull], [Dfull.T, None]], format="csr").astype(np.complex128)
    return A


def dirichlet_dofs(dir_nodes, dim):
    """All velocity components of every Dirichlet node (Eq. shape_fun: eta_g)."""
    dn = np.asarray(dir_nodes, dtype=np.int64)
    return (dn[:, None] * dim + np.arange(dim)[None, :]).ravel()


def lifted_system(A, dir_dofs, g_flat):
    """Split A into free/Dirichlet parts and lift the prescribed values:
    returns (A_FF, b_F, free) with b_F = -A_FD g (zero Neumann data; both the
    momentum and the continuity rows receive their lift)."""
    n = A.shape[0]
    is_dir = np.zeros(n, dtype=bool)
    is_dir[dir_dofs] = True
    free = np.flatnonzero(~is_dir)
    A_FF = A[free][:, free]
    A_FD = A[free][:, dir_dofs]
    b_F = -(A_FD @ g_flat)
    return A_FF.tocsc(), b_F, free


def direct_solve(A_FF, b_F):
    """Sparse LU (SuperLU) of one lifted system.  The minimum-degree ordering
    of A + A^T suits the symmetric saddle-point structure; SuperLU's default
    column ordering fills in several times more on these systems."""
    lu = sla.splu(A_FF, permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.1,
                  options=dict(SymmetricMode=True))
    return lu.solve(b_F)


def solve_modes(mats, wl):
    """Exact solution of every mode (sparse LU per mode, complex128).

    Returns X [m][n] in the full dof ordering with X_D = g."""
    d = mats["dim"]
    dd = dirichlet_dofs(wl["dir_nodes"], d)
    n = dof_count(mats)
    X = np.zeros((len(wl["omegas"]), n), dtype=np.complex128)
    for k, w in enumerate(wl["omegas"]):
        A = saddle_matrix(mats, w, wl["rho"], wl["mu"])
        g = wl["g"][k].reshape(-1)
        A_FF, b_F, free = lifted_system(A, dd, g)
        b_F = b_F + _load(mats, wl, k)[free]
        X[k, dd] = g
        if np.any(b_F != 0):
            X[k, free] = direct_solve(A_FF, b_F)
    return X


def _load(mats, wl, k):
    """Full-length momentum load of mode k: the Neumann term int_{Gamma_h} M_A h_c
    (wl["load"] [m][N][d], e.g. from oracle.boundary.neumann_load), zero if absent."""
    n = dof_count(mats)
    out = np.zeros(n, dtype=np.complex128)
    if wl.get("load") is not None:
        out[: mats["dim"] * mats["N"]] = np.asarray(wl["load"][k]).reshape(-1)
    return out


def masked_apply(mats, omegas, rho, mu, dir_nodes, Xblock):
    """y_k = A_hat(omega_k) x_k for every mode: Dirichlet velocity rows return
    x unchanged, every other row multiplies by A with the Dirichlet columns
    removed.  Xblock is [n][m] (mode-interleaved); returns [n][m]."""
    d = mats["dim"]
    dd = dirichlet_dofs(dir_nodes, d)
    n = dof_count(mats)
    mask = np.ones(n)
    mask[dd] = 0.0
    Y = np.empty_like(Xblock)
    for k, w in enumerate(omegas):
        A = saddle_matrix(mats, w, rho, mu)
        x = Xblock[:, k]
        y = mask * (A @ (mask * x))
        y[dd] = x[dd]
        Y[:, k] = y
    return Y


def rhs_block(mats, wl):
    """Lifted right-hand side of every mode, full length: b_F = -A_FD g on
    free rows, b_D = g on Dirichlet rows.  Returns [n][m]."""
    d = mats["dim"]
    dd = dirichlet_dofs(wl["dir_nodes"], d)
    n = dof_count(mats)
    B = np.zeros((n, len(wl["omegas"])), dtype=np.complex128)
    for k, w in enumerate(wl["omegas"]):
        A = saddle_matrix(mats, w, wl["rho"], wl["mu"])
        g = wl["g"][k].reshape(-1)
        gfull = np.zeros(n, dtype=np.complex128)
        gfull[dd] = g
        b = -(A @ gfull) + _load(mats, wl, k)
        b[dd] = g
        B[:, k] = b
    return B


def relative_residual(mats, wl, X):
    """||b_F - A_FF x_F - A_FD g|| / ||b_F|| per mode (Eq. ls_error over the
    unknowns of Eq. linear_sys_def, i.e. the non-Dirichlet dofs)."""
    d = mats["dim"]
    dd = dirichlet_dofs(wl["dir_nodes"], d)
    out = []
    for k, w in enumerate(wl["omegas"]):
        A = saddle_matrix(mats, w, wl["rho"], wl["mu"])
        g = wl["g"][k].reshape(-1)
        A_FF, b_F, free = lifted_system(A, dd, g)
        b_F = b_F + _load(mats, wl, k)[free]
        r = b_F - A_FF @ X[k, free]
        nb = np.linalg.norm(b_F)
        out.append(np.linalg.norm(r) / nb if nb > 0 else np.linalg.norm(r))
    return np.array(out)


# -------------------------------------------------------- post-processing

def split_fields(mats, x):
    """Full dof vector -> velocity [N][d], pressure [P]."""
    d, N = mats["dim"], mats["N"]
    return x[: d * N].reshape(N, d), x[d * N:]


def reconstruct(Umodes, omegas, n_t, period):
    """u(t_s) = Re sum_k U_k e^{j omega_k t_s}, t_s = s T / n_t (Eq. sol_reconstruct
    with real physical fields).  Umodes [m][...] complex; returns [n_t][...]."""
    t = np.arange(n_t) * (period / n_t)
    out = np.zeros((n_t,) + Umodes.shape[1:], dtype=np.float64)
    for s in range(n_t):
        acc = np.zeros(Umodes.shape[1:], dtype=np.complex128)
        for k, w in enumerate(omegas):
            acc += Umodes[k] * np.exp(1j * w * t[s])
        out[s] = acc.real
    return out


def l2_norm(Ms, u):
    """||u||_{L2(Omega)} of a nodal P2 vector field u [N][d] via M_s."""
    u = np.asarray(u)
    if u.ndim == 1:
        u = u[:, None]
    tot = 0.0
    for c in range(u.shape[1]):
        tot += np.real(np.vdot(u[:, c], Ms @ u[:, c]))
    return np.sqrt(max(tot, 0.0))


def relative_l2_error(Ms, u_ref, u_h):
    """e = ||u - u^h|| / ||u|| (Eq. total_error)."""
    return l2_norm(Ms, np.asarray(u_ref) - np.asarray(u_h)) / l2_norm(Ms, u_ref)
