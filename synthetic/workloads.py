"""Seeded workloads shaped like the paper's channel and pipe cases.

A workload is a mesh (``synthetic.meshes``) plus physics (rho, mu, period T),
the mode frequencies omega_k = 2 pi k / T (Eq. vaptransform) and the
Dirichlet data of every mode on every Dirichlet node: zero on walls, c_k times
the analytic fully developed profile on the inlet.  Boundary data are defined
so that the physical field is Re sum_k c_k g_k(x) e^{j omega_k t}.

Dirichlet nodes are the nodes tagged WALL or INLET, in ascending node id; the
outlet is traction-free (natural boundary, zero Neumann data).
"""
from __future__ import annotations

import numpy as np

from . import meshes
from .womersley import channel_profile, pipe_profile


def dirichlet_nodes(tag):
    return np.flatnonzero((tag & (meshes.WALL | meshes.INLET)) != 0).astype(np.int64)


def phases(n_modes, seed=0):
    """c_0 = 1, c_k = k^-2 exp(j phi_k), phi_k ~ U[0, 2 pi) (numpy PCG64, seed)."""
    rng = np.random.default_rng(seed)
    phi = rng.uniform(0.0, 2.0 * np.pi, size=n_modes)
    k = np.arange(n_modes, dtype=np.float64)
    c = np.empty(n_modes, dtype=np.complex128)
    c[0] = 1.0
    c[1:] = k[1:] ** -2.0 * np.exp(1j * phi[1:])
    return c


def _inlet_values(mesh, omegas, coeffs, rho, mu, G):
    tag = mesh["tag"]
    xyz = mesh["xyz"]
    dn = dirichlet_nodes(tag)
    d = mesh["dim"]
    g = np.zeros((len(omegas), dn.size, d), dtype=np.complex128)
    inl = ((tag[dn] & meshes.INLET) != 0) & ((tag[dn] & meshes.WALL) == 0)
    pts = xyz[dn[inl]]
    for k, (w, c) in enumerate(zip(omegas, coeffs)):
        if d == 2:
            prof = channel_profile(pts[:, 1], w, mesh["half_height"], rho, mu, G)
        else:
            r = np.hypot(pts[:, 1], pts[:, 2])
            prof = pipe_profile(r, w, mesh["radius"], rho, mu, G)
        g[k, inl, 0] = c * prof
    return dn, g


def channel_workload(nx=32, ny=8, n_modes=8, rho=1.0, mu=0.01, period=1.0, G=1.0):
    """Womersley channel [0,4]x[-0.5,0.5], c_k = 1 for all modes."""
    mesh = meshes.channel2d(nx, ny)
    omegas = 2.0 * np.pi * np.arange(n_modes) / period
    coeffs = np.ones(n_modes, dtype=np.complex128)
    dn, g = _inlet_values(mesh, omegas, coeffs, rho, mu, G)
    return dict(mesh=mesh, rho=rho, mu=mu, period=period, G=G, omegas=omegas,
                coeffs=coeffs, dir_nodes=dn, g=g, name=f"womersley channel {nx}x{ny}, {n_modes} modes")


# viscosity that puts the pipe's Womersley numbers W_k = omega_k R^2 rho/mu at
# 20 k / 31, i.e. in [0.65, 20] for k = 1..31 with R = rho = T = 1
PIPE_MU = 2.0 * np.pi * 31.0 / 20.0


def pipe_workload(n_c=8, n_r=6, n_x=71, n_modes=32, radius=1.0, length=10.0, rho=1.0,
                  mu=PIPE_MU, period=1.0, G=1.0, jitter=0.05, seed=0, stenosis=0.0, curved=False):
    """Jittered O-grid pipe; c_k = k^-2 exp(j phi_k) with seeded phases
    (``curved``: wall edge nodes projected onto the wall)."""
    mesh = meshes.pipe3d(radius=radius, length=length, n_c=n_c, n_r=n_r, n_x=n_x,
                         jitter=jitter, seed=seed, stenosis=stenosis, curved=curved)
    omegas = 2.0 * np.pi * np.arange(n_modes) / period
    coeffs = phases(n_modes, seed)
    dn, g = _inlet_values(mesh, omegas, coeffs, rho, mu, G)
    return dict(mesh=mesh, rho=rho, mu=mu, period=period, G=G, omegas=omegas,
                coeffs=coeffs, dir_nodes=dn, g=g,
                name=f"womersley pipe N={mesh['xyz'].shape[0]}, {n_modes} modes")


def bifurcation_workload(h=0.2, n_modes=16, rho=1.0, mu=PIPE_MU, period=1.0, G=1.0, seed=0, **geom):
    """Stenosed bifurcation (``meshes.bifurcation3d``) with the pipe's physics:
    Womersley inlet profile of the unit-radius parent (node radius clipped to
    the parent radius), c_k = k^-2 exp(j phi_k) with seeded phases, no-slip
    walls, traction-free daughter outlets."""
    mesh = meshes.bifurcation3d(h=h, **geom)
    omegas = 2.0 * np.pi * np.arange(n_modes) / period
    coeffs = phases(n_modes, seed)
    tag = mesh["tag"]
    dn = dirichlet_nodes(tag)
    g = np.zeros((n_modes, dn.size, 3), dtype=np.complex128)
    inl = ((tag[dn] & meshes.INLET) != 0) & ((tag[dn] & meshes.WALL) == 0)
    pts = mesh["xyz"][dn[inl]]
    r = np.minimum(np.hypot(pts[:, 1], pts[:, 2]), mesh["radius"])
    for k, (w, c) in enumerate(zip(omegas, coeffs)):
        g[k, inl, 0] = c * pipe_profile(r, w, mesh["radius"], rho, mu, G)
    return dict(mesh=mesh, rho=rho, mu=mu, period=period, G=G, omegas=omegas, coeffs=coeffs, dir_nodes=dn, g=g,
                name=f"stenosed bifurcation N={mesh['xyz'].shape[0]}, {n_modes} modes")


def exact_nodal(wl, k):
    """Analytic (u, p) of mode k at the nodes: velocity [N][d], pressure [P].

    Valid for the straight channel; for the pipe it is the continuum solution
    (the polygonal wall makes the FE solution differ at O(h^2..h^3))."""
    mesh = wl["mesh"]
    xyz = mesh["xyz"]
    d = mesh["dim"]
    w, c = wl["omegas"][k], wl["coeffs"][k]
    u = np.zeros((xyz.shape[0], d), dtype=np.complex128)
    if d == 2:
        u[:, 0] = c * channel_profile(xyz[:, 1], w, mesh["half_height"], wl["rho"], wl["mu"], wl["G"])
    else:
        r = np.hypot(xyz[:, 1], xyz[:, 2])
        u[:, 0] = c * pipe_profile(r, w, mesh["radius"], wl["rho"], wl["mu"], wl["G"])
    P = mesh["n_vertices"]
    p = c * wl["G"] * (mesh["length"] - xyz[:P, 0]) + 0j
    return u, p


def random_block(n_dofs, n_modes, seed, dtype=np.complex128):
    """Seeded complex test block [n_dofs][n_modes] with entries ~ U(-1,1)+jU(-1,1)."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, size=(n_dofs, n_modes)) + 1j * rng.uniform(-1, 1, size=(n_dofs, n_modes))
    return x.astype(dtype)


def union_workload(wls):
    """Batch of workloads with equal physics and mode lists as one mesh of
    independent components: the union mesh, node->component map, and the
    union's Dirichlet data (ascending union node id)."""
    from .meshes import union
    mesh, node_comp, maps = union([w["mesh"] for w in wls])
    dn = dirichlet_nodes(mesh["tag"])
    pos = {int(n): i for i, n in enumerate(dn)}
    m = len(wls[0]["omegas"])
    d = mesh["dim"]
    g = np.zeros((m, dn.size, d), dtype=np.complex128)
    for w, mp in zip(wls, maps):
        idx = np.array([pos[int(mp[n])] for n in w["dir_nodes"]], dtype=np.int64)
        g[:, idx, :] = w["g"]
    return dict(mesh=mesh, node_comp=node_comp, n_comp=len(wls), maps=maps, parts=wls, rho=wls[0]["rho"],
                mu=wls[0]["mu"], period=wls[0]["period"], omegas=wls[0]["omegas"], dir_nodes=dn, g=g,
                name=f"batch of {len(wls)} pipes")


def uneven_pipes(n_meshes=48, n_modes=16, seed=0, n_min=20_000, n_max=400_000, scale=1.0):
    """Seeded batch of stenosed pipes of uneven size: R ~ U[0.5, 1.5],
    L ~ U[5, 20], s ~ U[0, 0.5], target P2 node count log-uniform in
    [n_min, n_max] (times `scale`); phases of c_k drawn per mesh."""
    from .meshes import pipe_size
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_meshes):
        R = rng.uniform(0.5, 1.5)
        L = rng.uniform(5.0, 20.0)
        s = rng.uniform(0.0, 0.5)
        target = np.exp(rng.uniform(np.log(n_min), np.log(n_max))) * scale
        best = None
        for n_c in range(2, 40):
            n_r = max(1, int(round(0.75 * n_c)))
            hc = 2 * 0.5 * R / n_c
            n_x = max(2, int(round(L / (1.1 * hc))))
            N, _ = pipe_size(n_c, n_r, n_x)
            if best is None or abs(np.log(N / target)) < abs(np.log(best[0] / target)):
                best = (N, n_c, n_r, n_x)
        _, n_c, n_r, n_x = best
        wl = pipe_workload(n_c=n_c, n_r=n_r, n_x=n_x, n_modes=n_modes, radius=R, length=L, stenosis=s,
                           seed=seed + 1 + i)
        out.append(wl)
    return out


def traction_inlet(mesh, omegas, hx, rho, mu, neumann_tag):
    """The paper's validation setting (Sec. 3.2 channel, Sec. 3.4 pipe): the
    inlet carries a uniform streamwise traction h = (hx, 0[, 0]) for every mode
    (a cosine in time for omega > 0) instead of a velocity, the walls are
    no-slip and the outlet traction-free.  Inlet nodes are retagged with
    `neumann_tag` (wall nodes stay Dirichlet); returns the workload with zero
    Dirichlet data and the nodal tractions h [m][N][d] (input data only: the
    boundary integral is the solver's or the oracle's business)."""
    tag = mesh["tag"].copy()
    inl = (tag & meshes.INLET) != 0
    tag[inl] = (tag[inl] & ~np.uint8(meshes.INLET)) | np.uint8(neumann_tag)
    mesh = dict(mesh, tag=tag)
    d = mesh["dim"]
    walls = np.flatnonzero((tag & meshes.WALL) != 0)
    N = mesh["xyz"].shape[0]
    m = len(omegas)
    h = np.zeros((m, N, d), dtype=np.complex128)
    h[:, :, 0] = hx
    return dict(mesh=mesh, omegas=np.asarray(omegas, dtype=np.float64), rho=rho, mu=mu, dir_nodes=walls,
                g=np.zeros((m, walls.size, d), dtype=np.complex128), h=h, hx=hx)


def paper_channel(omegas, rho=1.0, mu=0.01, hx=1.0, neumann_tag=8):
    """The paper's 2D channel (Sec. 3.2): aspect ratio 5, 882 P2 triangles,
    1,881 nodes and 4,262 dofs, i.e. 49 x 9 quads of [0, 5] x [-0.5, 0.5]
    split in two; traction inlet."""
    mesh = meshes.channel2d(49, 9, length=5.0, half_height=0.5)
    return traction_inlet(mesh, omegas, hx, rho, mu, neumann_tag)


def paper_pipe(target_nodes, omegas, rho=1.0, mu=1.0, hx=1.0, neumann_tag=8, seed=0, curved=True):
    """The paper's pipe (Sec. 3.4): L/R = 15, R = 1, traction inlet, on an
    O-grid mesh of about target_nodes P2 nodes (QM1-QM4: 37,469 / 70,872 /
    133,645 / 225,610 nodes), no jitter; wall edge nodes on the cylinder
    (``curved``, the paper's node projection) or at chord midpoints."""
    mesh = meshes.pipe_for_nodes(target_nodes, radius=1.0, length=15.0, jitter=0.0, seed=seed, curved=curved)
    return traction_inlet(mesh, omegas, hx, rho, mu, neumann_tag)


def curved_channel(n_r, n_t, curved=True, mu=1.0, K=1.0, r1=1.0, r2=2.0, theta=0.5 * np.pi, neumann_tag=8):
    """Steady Stokes flow in the annular sector r1 <= r <= r2, 0 <= t <= theta
    (meshes.annulus2d) driven by the azimuthal pressure p = K (theta - t):
    u = u_t(r) e_t with u_t = A r + B / r - K / (2 mu) r ln r, u_t(r1) = u_t(r2) = 0.
    Dirichlet data on the inlet and the walls; the outlet nodes also carry
    ``neumann_tag`` with the exact pseudo-traction (-p I + mu grad u) n =
    -mu u_t / r e_r there.  Returns the workload, the nodal tractions h [1][N][2]
    and the exact nodal velocity."""
    m = meshes.annulus2d(n_r=n_r, n_t=n_t, r1=r1, r2=r2, theta=theta, curved=curved)
    c = K / (2.0 * mu)
    A = c * (r2 * np.log(r2) - r1 * r1 / r2 * np.log(r1)) / (r2 - r1 * r1 / r2)
    B = c * r1 * r1 * np.log(r1) - A * r1 * r1
    xyz = m["xyz"]
    r = np.hypot(xyz[:, 0], xyz[:, 1])
    t = np.arctan2(xyz[:, 1], xyz[:, 0])
    ut = A * r + B / r - c * r * np.log(r)
    uex = np.stack([-np.sin(t) * ut, np.cos(t) * ut], axis=1)
    tag = m["tag"].copy()
    out = (tag & meshes.OUTLET) != 0
    tag[out] |= np.uint8(neumann_tag)
    m = dict(m, tag=tag)
    dn = dirichlet_nodes(tag)
    h = np.zeros((1,) + xyz.shape, dtype=np.complex128)
    h[0, :, 0] = -mu * ut / r * np.cos(theta)
    h[0, :, 1] = -mu * ut / r * np.sin(theta)
    wl = dict(mesh=m, omegas=np.array([0.0]), rho=1.0, mu=mu, dir_nodes=dn,
              g=uex[dn][None].astype(np.complex128), h=h, name=f"curved channel {n_r}x{n_t}")
    return wl, uex
