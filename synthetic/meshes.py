"""Seeded synthetic P2 meshes: the shared *input* of the oracle and the CUDA path.

Nothing here computes any part of the finite-element method (no shape
functions, no integrals, no matrices).  The generators only place vertices,
form simplices, insert straight-sided P2 edge nodes at edge midpoints and tag
boundary nodes, i.e. they produce the mesh a user would hand to the solver.

Conventions (the paper uses P2 velocity / P1 pressure simplices, Sec. 2.3):
  * ``xyz``   float64 [N][d]  node coordinates
  * ``conn``  int32   [E][6|10]  P2 connectivity in VTK order: the simplex
    vertices, then the edge nodes (0,1),(1,2),(2,0)[,(0,3),(1,3),(2,3)]
  * vertex nodes are numbered first (ids 0..P-1), so the P1 pressure dof of a
    vertex is its node id
  * ``tag``   uint8   [N]  bit flags WALL=1, INLET=2, OUTLET=4 (a node may
    carry several; corner nodes on a wall and the inlet carry both)
The streamwise direction is x in both the channel and the pipe.
"""
from __future__ import annotations

import numpy as np

WALL, INLET, OUTLET = 1, 2, 4

# VTK quadratic-simplex edge order (local vertex pairs)
TRI_EDGES = ((0, 1), (1, 2), (2, 0))
TET_EDGES = ((0, 1), (1, 2), (2, 0), (0, 3), (1, 3), (2, 3))


def _orient_positive(vxyz, simp):
    """Swap local vertices 1,2 of simplices with negative signed measure."""
    d = simp.shape[1] - 1
    x0 = vxyz[simp[:, 0]]
    J = np.stack([vxyz[simp[:, i + 1]] - x0 for i in range(d)], axis=-1)
    det = np.linalg.det(J)
    if np.any(det == 0.0):
        raise ValueError("degenerate simplex in generator")
    neg = det < 0
    simp = simp.copy()
    simp[neg, 1], simp[neg, 2] = simp[neg, 2].copy(), simp[neg, 1].copy()
    return simp


def _add_p2_nodes(vxyz, simp, edge_sort_key):
    """Insert one node at the midpoint of every unique simplex edge.

    ``edge_sort_key(lo, hi, mid_xyz)`` returns a lexsort key tuple (last key is
    primary, numpy.lexsort convention) that fixes the numbering of the edge
    nodes; vertex ids are kept, edge nodes follow them.
    """
    P = vxyz.shape[0]
    d = simp.shape[1] - 1
    edges = TRI_EDGES if d == 2 else TET_EDGES
    a = np.stack([simp[:, i] for i, _ in edges], axis=1).astype(np.int64)
    b = np.stack([simp[:, j] for _, j in edges], axis=1).astype(np.int64)
    lo = np.minimum(a, b).ravel()
    hi = np.maximum(a, b).ravel()
    key = lo * P + hi
    ukey, inv = np.unique(key, return_inverse=True)
    ulo = ukey // P
    uhi = ukey % P
    mid = 0.5 * (vxyz[ulo] + vxyz[uhi])
    order = np.lexsort(edge_sort_key(ulo, uhi, mid))
    rank = np.empty_like(order)
    rank[order] = np.arange(order.size)
    edge_id = P + rank[inv].reshape(a.shape)
    xyz = np.concatenate([vxyz, mid[order]], axis=0)
    conn = np.concatenate([simp.astype(np.int64), edge_id], axis=1).astype(np.int32)
    edge_ends = np.stack([ulo[order], uhi[order]], axis=1)
    return xyz, conn, edge_ends


def channel2d(nx=32, ny=8, length=4.0, half_height=0.5):
    """Structured P2 triangulation of [0,length] x [-H,H].

    Every quad (i,j) is cut along its (i,j)->(i+1,j+1) diagonal.  P2 nodes lie
    on the (2nx+1) x (2ny+1) lattice; vertices are numbered first in x-fastest
    lattice order, then the remaining lattice nodes in x-fastest order.
    Walls y=+-H, inlet x=0, outlet x=length.
    """
    H = half_height
    I = np.arange(nx + 1)
    J = np.arange(ny + 1)
    vx = np.repeat(J[:, None], nx + 1, axis=1) * 0 + I[None, :]
    vy = np.repeat(J[:, None], nx + 1, axis=1)
    vxyz = np.stack([vx.ravel() * (length / nx), -H + vy.ravel() * (2 * H / ny)], axis=1)
    vid = lambda i, j: j * (nx + 1) + i
    tris = []
    for j in range(ny):
        for i in range(nx):
            v00, v10, v11, v01 = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
            tris.append((v00, v10, v11))
            tris.append((v00, v11, v01))
    simp = _orient_positive(vxyz, np.array(tris, dtype=np.int64))
    hx, hy = length / (2 * nx), 2 * H / (2 * ny)

    def key(lo, hi, mid):
        li = np.rint(mid[:, 0] / hx).astype(np.int64)
        lj = np.rint((mid[:, 1] + H) / hy).astype(np.int64)
        return (li, lj)  # lexsort: lj primary, li secondary -> x-fastest

    xyz, conn, _ = _add_p2_nodes(vxyz, simp, key)
    tag = np.zeros(xyz.shape[0], dtype=np.uint8)
    eps = 1e-12
    tag[np.abs(np.abs(xyz[:, 1]) - H) < eps] |= WALL
    tag[np.abs(xyz[:, 0]) < eps] |= INLET
    tag[np.abs(xyz[:, 0] - length) < eps] |= OUTLET
    return dict(dim=2, xyz=xyz, conn=conn, tag=tag, n_vertices=vxyz.shape[0],
                name=f"channel {nx}x{ny}", length=length, half_height=H)


def _structured_2d(vxyz, nx, ny):
    """Triangles of an (nx+1) x (ny+1) vertex lattice (x-fastest ids), every
    quad cut along its (i,j)->(i+1,j+1) diagonal, positively oriented."""
    vid = lambda i, j: j * (nx + 1) + i
    tris = []
    for j in range(ny):
        for i in range(nx):
            v00, v10, v11, v01 = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
            tris.append((v00, v10, v11))
            tris.append((v00, v11, v01))
    return _orient_positive(vxyz, np.array(tris, dtype=np.int64))


def _lattice_key(nx):
    def key(lo, hi, mid):
        # edge nodes numbered by their lattice position (i + i', j + j'), x-fastest
        i = lo % (nx + 1) + hi % (nx + 1)
        j = lo // (nx + 1) + hi // (nx + 1)
        return (i, j)
    return key


def annulus2d(n_r=4, n_t=16, r1=1.0, r2=2.0, theta=0.5 * np.pi, curved=True):
    """Annular sector r1 <= r <= r2, 0 <= t <= theta (a curved channel):
    vertices on the polar lattice, straight-sided P2 edge nodes at edge
    midpoints except, with ``curved``, those of edges on the circles r = r1 and
    r = r2, projected radially onto the circle (isoparametric boundary, the
    paper's Sec. 3.1 node projection).  Walls r = r1, r2; inlet t = 0; outlet
    t = theta."""
    rr = np.linspace(r1, r2, n_r + 1)
    tt = np.linspace(0.0, theta, n_t + 1)
    R, T = np.meshgrid(rr, tt, indexing="ij")  # [radius j][angle i]: ids angle-fastest
    R, T = R.ravel(), T.ravel()
    vxyz = np.stack([R * np.cos(T), R * np.sin(T)], axis=1)
    simp = _structured_2d(vxyz, n_t, n_r)
    xyz, conn, ends = _add_p2_nodes(vxyz, simp, _lattice_key(n_t))
    P = vxyz.shape[0]
    vr = np.hypot(vxyz[:, 0], vxyz[:, 1])
    vt = np.arctan2(vxyz[:, 1], vxyz[:, 0])
    eps = 1e-9
    vtag = np.zeros(P, dtype=np.uint8)
    vtag[(np.abs(vr - r1) < eps) | (np.abs(vr - r2) < eps)] |= WALL
    vtag[np.abs(vt) < eps] |= INLET
    vtag[np.abs(vt - theta) < eps] |= OUTLET
    tag = np.zeros(xyz.shape[0], dtype=np.uint8)
    tag[:P] = vtag
    ra, rb = vr[ends[:, 0]], vr[ends[:, 1]]
    same_circle = (np.abs(ra - rb) < eps) & ((np.abs(ra - r1) < eps) | (np.abs(ra - r2) < eps))
    same_ray = np.abs(vt[ends[:, 0]] - vt[ends[:, 1]]) < eps
    etag = np.zeros(ends.shape[0], dtype=np.uint8)
    etag[same_circle] |= WALL
    etag[same_ray] |= vtag[ends[same_ray, 0]] & vtag[ends[same_ray, 1]] & (INLET | OUTLET)
    tag[P:] = etag
    if curved:
        e = np.flatnonzero(same_circle) + P
        m = xyz[e]
        xyz[e] = m * (ra[same_circle] / np.hypot(m[:, 0], m[:, 1]))[:, None]
    return dict(dim=2, xyz=xyz, conn=conn, tag=tag, n_vertices=P, name=f"annulus {n_r}x{n_t}",
                r1=r1, r2=r2, theta=theta)


def nozzle_half_height(x, h_in=1.0, ratio=2.0, x1=2.0, x2=6.0):
    """Wall of the diverging nozzle: h_in up to x1, a cosine ramp to ratio * h_in at x2, then constant."""
    x = np.asarray(x, dtype=np.float64)
    s = np.clip((x - x1) / (x2 - x1), 0.0, 1.0)
    return h_in * (1.0 + (ratio - 1.0) * 0.5 * (1.0 - np.cos(np.pi * s)))


def nozzle2d(nx=30, ny=10, length=10.0, h_in=1.0, ratio=2.0, x1=2.0, x2=6.0):
    """2D diverging nozzle of expansion ratio 2 (the paper's Sec. 3.3): walls
    y = +-h(x), h from nozzle_half_height; vertices (x_i, eta_j h(x_i)) on an
    (nx+1) x (ny+1) lattice; P2 edge nodes at edge midpoints except the wall
    edge nodes, placed on the wall at the midpoint abscissa (the paper
    projects inserted boundary nodes onto the curved wall).  nx = 30, ny = 10
    gives the paper's 600 quadratic triangles and 1,281 nodes.  Inlet x = 0,
    outlet x = length."""
    xs = np.linspace(0.0, length, nx + 1)
    eta = np.linspace(-1.0, 1.0, ny + 1)
    X, E = np.meshgrid(xs, eta)  # rows: eta (j), columns: x (i) -> x-fastest
    H = nozzle_half_height(X, h_in, ratio, x1, x2)
    vxyz = np.stack([X.ravel(), (E * H).ravel()], axis=1)
    simp = _structured_2d(vxyz, nx, ny)
    xyz, conn, ends = _add_p2_nodes(vxyz, simp, _lattice_key(nx))
    P = vxyz.shape[0]
    vj = np.arange(P) // (nx + 1)
    vi = np.arange(P) % (nx + 1)
    vtag = np.zeros(P, dtype=np.uint8)
    vtag[(vj == 0) | (vj == ny)] |= WALL
    vtag[vi == 0] |= INLET
    vtag[vi == nx] |= OUTLET
    tag = np.zeros(xyz.shape[0], dtype=np.uint8)
    tag[:P] = vtag
    a, b = ends[:, 0], ends[:, 1]
    wall_e = ((vj[a] == 0) & (vj[b] == 0)) | ((vj[a] == ny) & (vj[b] == ny))
    end_e = ((vi[a] == 0) & (vi[b] == 0)) | ((vi[a] == nx) & (vi[b] == nx))
    tag[P:][wall_e] |= WALL
    tag[P:][end_e] |= vtag[a[end_e]] & vtag[b[end_e]] & (INLET | OUTLET)
    e = np.flatnonzero(wall_e) + P
    xm = xyz[e, 0]
    xyz[e, 1] = np.sign(xyz[e, 1]) * nozzle_half_height(xm, h_in, ratio, x1, x2)
    return dict(dim=2, xyz=xyz, conn=conn, tag=tag, n_vertices=P, name=f"nozzle {nx}x{ny}", length=length,
                h_in=h_in, ratio=ratio)


def _ogrid_section(n_c, n_r, radius, core=0.5):
    """5-block O-grid of the disk: a core square of half-width core*R and a
    ring of 4*n_c x n_r quads blending the square perimeter to the circle.
    Returns 2D vertex coords (y,z), quads (ccw), and a mask of circle vertices."""
    a = core * radius
    ii, jj = np.meshgrid(np.arange(n_c + 1), np.arange(n_c + 1))
    sq = np.stack([-a + 2 * a * ii.ravel() / n_c, -a + 2 * a * jj.ravel() / n_c], axis=1)
    sid = lambda i, j: j * (n_c + 1) + i
    nq = 4 * n_c
    per_id = np.empty(nq, dtype=np.int64)
    for q in range(nq):
        s, t = divmod(q, n_c)
        if s == 0:
            per_id[q] = sid(n_c, t)
        elif s == 1:
            per_id[q] = sid(n_c - t, n_c)
        elif s == 2:
            per_id[q] = sid(0, n_c - t)
        else:
            per_id[q] = sid(t, 0)
    theta = -np.pi / 4 + (np.pi / 2) * np.arange(nq) / n_c
    circ = radius * np.stack([np.cos(theta), np.sin(theta)], axis=1)
    ring = []
    for l in range(1, n_r + 1):
        rho = l / n_r
        ring.append((1 - rho) * sq[per_id] + rho * circ)
    vxy = np.concatenate([sq] + ring, axis=0)
    base = (n_c + 1) ** 2
    rid = lambda l, q: per_id[q % nq] if l == 0 else base + (l - 1) * nq + (q % nq)
    quads = []
    for j in range(n_c):
        for i in range(n_c):
            quads.append((sid(i, j), sid(i + 1, j), sid(i + 1, j + 1), sid(i, j + 1)))
    for l in range(1, n_r + 1):
        for q in range(nq):
            quads.append((rid(l - 1, q), rid(l, q), rid(l, q + 1), rid(l - 1, q + 1)))
    on_circle = np.zeros(vxy.shape[0], dtype=bool)
    on_circle[base + (n_r - 1) * nq:] = True
    if n_r == 0:
        raise ValueError("n_r must be >= 1")
    vxy[on_circle] = radius * vxy[on_circle] / np.linalg.norm(vxy[on_circle], axis=1)[:, None]
    return vxy, np.array(quads, dtype=np.int64), on_circle


def _split_quads(quads):
    """Cut each quad along the diagonal through its smallest vertex id."""
    tris = []
    for v in quads:
        k = int(np.argmin(v))
        if k % 2 == 0:
            tris.append((v[0], v[1], v[2]))
            tris.append((v[0], v[2], v[3]))
        else:
            tris.append((v[1], v[2], v[3]))
            tris.append((v[1], v[3], v[0]))
    return np.array(tris, dtype=np.int64)


def stenosis_radius(x, radius, s, x_c, ell):
    """Cosine stenosis R(x) = R0 [1 - (s/2)(1 + cos(2 pi (x - x_c)/ell))] for
    |x - x_c| <= ell/2, R0 elsewhere (s = fractional radius reduction)."""
    x = np.asarray(x, dtype=np.float64)
    r = np.full_like(x, radius)
    m = np.abs(x - x_c) <= ell / 2
    r[m] = radius * (1 - 0.5 * s * (1 + np.cos(2 * np.pi * (x[m] - x_c) / ell)))
    return r


def pipe3d(radius=1.0, length=10.0, n_c=8, n_r=6, n_x=71, jitter=0.05, seed=0,
           stenosis=0.0, core=0.5, curved=False):
    """Straight (optionally stenosed) round pipe along x, inlet x=0, outlet x=L.

    Cross-section: 5-block O-grid, each quad cut into 2 triangles; extruded in
    n_x layers; each prism (2D vertices a<b<c by id, bottom a,b,c / top
    a',b',c') is cut into the tets [a,b,c,a'], [b,c,a',b'], [c,a',b',c'] so
    that every vertical quad face is split by the same diagonal from both
    sides (the diagonal joins the bottom of the larger id to the top of the
    smaller) - a conforming 6-tet split of every hex.
    Interior vertices are jittered by U(-jitter, jitter) * h_local per axis
    (numpy PCG64, ``seed``), h_local = shortest incident edge.  Wall vertices
    stay on the (stenosed) circle, inlet/outlet vertices in their planes.
    A stenosis s > 0 scales each layer radially by R(x)/R0 (centre L/2,
    extent 4R0).  Node count N = (V2 + E2) (2 n_x + 1) with V2/E2 the 2D
    vertex/edge counts.  With ``curved`` the edge nodes of wall edges are
    projected radially onto the (stenosed) wall, so boundary elements are
    isoparametric (the paper's Sec. 3.1 node projection); otherwise every
    edge node is an edge midpoint.
    """
    vxy, quads, on_circle = _ogrid_section(n_c, n_r, radius, core)
    tris = _split_quads(quads)
    V2 = vxy.shape[0]
    xs = np.linspace(0.0, length, n_x + 1)
    vxyz = np.zeros(((n_x + 1) * V2, 3))
    for k, x in enumerate(xs):
        vxyz[k * V2:(k + 1) * V2, 0] = x
        vxyz[k * V2:(k + 1) * V2, 1:] = vxy
    tets = []
    ts = np.sort(tris, axis=1)
    for k in range(n_x):
        lo, hi = k * V2, (k + 1) * V2
        a, b, c = ts[:, 0], ts[:, 1], ts[:, 2]
        tets.append(np.stack([lo + a, lo + b, lo + c, hi + a], axis=1))
        tets.append(np.stack([lo + b, lo + c, hi + a, hi + b], axis=1))
        tets.append(np.stack([lo + c, hi + a, hi + b, hi + c], axis=1))
    simp = np.concatenate(tets, axis=0)
    wall_v = np.tile(on_circle, n_x + 1)
    layer = np.repeat(np.arange(n_x + 1), V2)
    inlet_v = layer == 0
    outlet_v = layer == n_x
    if stenosis > 0.0:
        rx = stenosis_radius(vxyz[:, 0], radius, stenosis, 0.5 * length, 4.0 * radius)
        vxyz[:, 1:] *= (rx / radius)[:, None]
    if jitter > 0.0:
        # shortest incident edge per vertex over the tets' 6 edges
        h = np.full(vxyz.shape[0], np.inf)
        for i, j in TET_EDGES:
            el = np.linalg.norm(vxyz[simp[:, i]] - vxyz[simp[:, j]], axis=1)
            np.minimum.at(h, simp[:, i], el)
            np.minimum.at(h, simp[:, j], el)
        rng = np.random.default_rng(seed)
        disp = rng.uniform(-jitter, jitter, size=vxyz.shape) * h[:, None]
        free = ~(wall_v | inlet_v | outlet_v)
        vxyz[free] += disp[free]
    simp = _orient_positive(vxyz, simp)
    n_layers = 2 * n_x

    def key(lo, hi, mid):
        # P2 layer of the midpoint (2k or 2k+1), then vertex ids
        pl = (lo // V2) + (hi // V2)
        return (hi, lo, pl)

    xyz, conn, ends = _add_p2_nodes(vxyz, simp, key)
    P = vxyz.shape[0]
    N = xyz.shape[0]
    tag = np.zeros(N, dtype=np.uint8)
    vtag = np.zeros(P, dtype=np.uint8)
    vtag[wall_v] |= WALL
    vtag[inlet_v] |= INLET
    vtag[outlet_v] |= OUTLET
    tag[:P] = vtag
    # an edge node lies on a boundary face iff both of its ends do: in this
    # O-grid no interior edge joins two wall vertices (n_r >= 1) and no edge
    # joins two vertices of an end plane except in that plane
    tag[P:] = vtag[ends[:, 0]] & vtag[ends[:, 1]]
    if curved:
        e = np.flatnonzero(tag[P:] & WALL) + P
        rw = radius if stenosis <= 0.0 else stenosis_radius(xyz[e, 0], radius, stenosis, 0.5 * length, 4.0 * radius)
        rr = np.hypot(xyz[e, 1], xyz[e, 2])
        xyz[e, 1:] *= (rw / rr)[:, None]
    assert n_layers >= 2
    return dict(dim=3, xyz=xyz, conn=conn, tag=tag, n_vertices=P,
                name=f"pipe R={radius} L={length} n_c={n_c} n_r={n_r} n_x={n_x} s={stenosis}",
                radius=radius, length=length, stenosis=stenosis)


def pipe_size(n_c, n_r, n_x):
    """(N, P) of pipe3d without building it (same counts as the generator)."""
    V2 = (n_c + 1) ** 2 + 4 * n_c * n_r
    T2 = 2 * (n_c * n_c + 4 * n_c * n_r)
    E2 = V2 + T2 - 1
    return (V2 + E2) * (2 * n_x + 1), V2 * (n_x + 1)


def pipe_for_nodes(target_nodes, radius=1.0, length=10.0, **kw):
    """Pick (n_c, n_r, n_x) so that N is close to target_nodes with cells of
    comparable size in the section and along the axis."""
    best = None
    for n_c in range(2, 64):
        n_r = max(1, int(round(0.75 * n_c)))
        hc = 2 * 0.5 * radius / n_c
        n_x = max(1, int(round(length / (1.1 * hc))))
        N, _ = pipe_size(n_c, n_r, n_x)
        if best is None or abs(np.log(N / target_nodes)) < abs(np.log(best[0] / target_nodes)):
            best = (N, n_c, n_r, n_x)
    _, n_c, n_r, n_x = best
    return pipe3d(radius=radius, length=length, n_c=n_c, n_r=n_r, n_x=n_x, **kw)


def union(mesh_list):
    """Disjoint union of P2 meshes of one dimension as one mesh.

    Vertices of every component come first (component order), then the edge
    nodes (component order), so the union keeps the vertex-first numbering.
    Returns (mesh, node_comp, maps) with maps[i][v] = union id of node v of
    component i."""
    dim = mesh_list[0]["dim"]
    Ps = [m["n_vertices"] for m in mesh_list]
    Ns = [m["xyz"].shape[0] for m in mesh_list]
    Ptot = sum(Ps)
    vbase = np.cumsum([0] + Ps[:-1])
    ebase = np.cumsum([0] + [n - p for n, p in zip(Ns, Ps)][:-1])
    Ntot = sum(Ns)
    xyz = np.zeros((Ntot, dim))
    tag = np.zeros(Ntot, dtype=np.uint8)
    node_comp = np.zeros(Ntot, dtype=np.int32)
    conns, maps = [], []
    for i, m in enumerate(mesh_list):
        v = np.arange(Ns[i])
        mp = np.where(v < Ps[i], vbase[i] + v, Ptot + ebase[i] + (v - Ps[i]))
        xyz[mp] = m["xyz"]
        tag[mp] = m["tag"]
        node_comp[mp] = i
        conns.append(mp[m["conn"]].astype(np.int32))
        maps.append(mp)
    mesh = dict(dim=dim, xyz=xyz, conn=np.concatenate(conns, axis=0), tag=tag, n_vertices=Ptot,
                name=f"union of {len(mesh_list)} meshes")
    return mesh, node_comp, maps


# Kuhn split of the unit cube: one tet per axis permutation, all sharing the
# main diagonal v000-v111; on every face the split diagonal joins the face's
# lowest and highest corner, so neighbouring cubes split shared faces alike.
_KUHN_PERMS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))


def bifurcation_inside(p, parent_len, stenosis, daughter_radius, daughter_len, angle_deg, radius=1.0):
    """Inside test of the bifurcation: stenosed parent x in [0, L_p] (cosine
    stenosis centred at L_p/2, extent 4R), a ball of radius R at the branch
    point (L_p, 0, 0), and two daughters of radius R_d and length L_d whose
    axes leave the branch point at +-angle in the x-y plane.  Returns
    (inside, (t+, r+), (t-, r-)) with the daughters' axial and radial
    coordinates."""
    x, y, z = p[..., 0], p[..., 1], p[..., 2]
    rp = np.hypot(y, z)
    inside = (x >= 0) & (x <= parent_len) & (rp <= stenosis_radius(x, radius, stenosis, 0.5 * parent_len,
                                                                  4.0 * radius))
    q = p - np.array([parent_len, 0.0, 0.0])
    inside |= np.einsum("...i,...i->...", q, q) <= radius * radius
    a = np.deg2rad(angle_deg)
    coords = []
    for sgn in (1.0, -1.0):
        d = np.array([np.cos(a), sgn * np.sin(a), 0.0])
        t = q @ d
        r = np.linalg.norm(q - t[..., None] * d, axis=-1)
        inside |= (t >= 0) & (t <= daughter_len) & (r <= daughter_radius)
        coords.append((t, r))
    return inside, coords[0], coords[1]


def bifurcation3d(h=0.2, parent_len=8.0, stenosis=0.5, daughter_radius=0.7, daughter_len=6.0, angle_deg=45.0,
                  radius=1.0):
    """Stenosed bifurcation on a voxel grid of spacing h: every cell whose
    centre is inside (``bifurcation_inside``) is kept and cut into the 6 Kuhn
    tets (conforming).  Boundary faces of kept cells are tagged from the
    cell beyond them: INLET if it lies at x < 0, OUTLET if it lies past the
    end of a daughter (axial t > L_d, radial r <= R_d), WALL otherwise.  A
    node carries the tags of every boundary face it lies on (vertices: the 4
    corners; edge nodes: the 4 sides and the split diagonal).  The wall is a
    staircase at resolution h.  About 7.6 P2 nodes per vertex; h = 0.038
    gives ~6M P2 nodes."""
    a = np.deg2rad(angle_deg)
    L_d = daughter_len
    tip = np.array([parent_len, 0.0, 0.0]) + (L_d + daughter_radius) * np.array([np.cos(a), np.sin(a), 0.0])
    hi = np.array([tip[0] + daughter_radius, max(tip[1] + daughter_radius, radius), radius])
    lo = np.array([0.0, -hi[1], -radius])
    n = np.ceil((hi - lo) / h).astype(np.int64) + 1
    lo[1] = -0.5 * n[1] * h   # symmetric in y and z about the axis
    lo[2] = -0.5 * n[2] * h
    ci = [lo[d] + (np.arange(n[d]) + 0.5) * h for d in range(3)]
    cx, cy, cz = np.meshgrid(ci[0], ci[1], ci[2], indexing="ij")
    cen = np.stack([cx, cy, cz], axis=-1)
    keep, _, _ = bifurcation_inside(cen, parent_len, stenosis, daughter_radius, L_d, angle_deg, radius)
    # vertices of kept cells, numbered x-major (streamwise), then y, then z
    vused = np.zeros(n + 1, dtype=bool)
    for o in np.ndindex(2, 2, 2):
        vused[o[0]:o[0] + n[0], o[1]:o[1] + n[1], o[2]:o[2] + n[2]] |= keep
    vid = -np.ones(n + 1, dtype=np.int64)
    vid[vused] = np.arange(int(vused.sum()))
    gi = np.argwhere(vused)
    vxyz = lo + gi * h
    cells = np.argwhere(keep)
    corner = lambda off: vid[cells[:, 0] + off[0], cells[:, 1] + off[1], cells[:, 2] + off[2]]
    tets = []
    for perm in _KUHN_PERMS:
        off = np.zeros(3, dtype=np.int64)
        ids = [corner(off)]
        for ax in perm:
            off = off.copy()
            off[ax] = 1
            ids.append(corner(off))
        tets.append(np.stack(ids, axis=1))
    simp = _orient_positive(vxyz, np.concatenate(tets, axis=0))

    def key(lo_, hi_, mid):
        return (lo_, hi_)

    xyz, conn, ends = _add_p2_nodes(vxyz, simp, key)
    P = vxyz.shape[0]
    N = xyz.shape[0]
    ekey = ends[:, 0] * P + ends[:, 1]
    eorder = np.argsort(ekey)
    tag = np.zeros(N, dtype=np.uint8)
    for ax in range(3):
        for side in (0, 1):
            # kept cells whose neighbour across the face (ax, side) is not kept
            nb = np.zeros_like(keep)
            sl_dst = [slice(None)] * 3
            sl_src = [slice(None)] * 3
            if side == 1:
                sl_dst[ax] = slice(0, n[ax] - 1)
                sl_src[ax] = slice(1, n[ax])
            else:
                sl_dst[ax] = slice(1, n[ax])
                sl_src[ax] = slice(0, n[ax] - 1)
            nb[tuple(sl_dst)] = keep[tuple(sl_src)]
            fc = np.argwhere(keep & ~nb)
            if fc.size == 0:
                continue
            outc = lo + (fc + 0.5) * h
            outc[:, ax] += (h if side == 1 else -h)
            _, (tp, rp_), (tm, rm) = bifurcation_inside(outc, parent_len, stenosis, daughter_radius, L_d,
                                                       angle_deg, radius)
            ftag = np.full(fc.shape[0], WALL, dtype=np.uint8)
            ftag[((tp > L_d) & (rp_ <= daughter_radius)) | ((tm > L_d) & (rm <= daughter_radius))] = OUTLET
            ftag[outc[:, 0] < 0] = INLET
            b, c = [d for d in range(3) if d != ax]
            cv = {}
            for ob in (0, 1):
                for oc in (0, 1):
                    off = np.zeros(3, dtype=np.int64)
                    off[ax] = side
                    off[b] = ob
                    off[c] = oc
                    cv[ob, oc] = vid[fc[:, 0] + off[0], fc[:, 1] + off[1], fc[:, 2] + off[2]]
            for v in cv.values():
                np.bitwise_or.at(tag, v, ftag)
            for (p0, p1) in (((0, 0), (1, 0)), ((1, 0), (1, 1)), ((1, 1), (0, 1)), ((0, 1), (0, 0)),
                             ((0, 0), (1, 1))):
                u, w = cv[p0], cv[p1]
                k = np.minimum(u, w) * P + np.maximum(u, w)
                pos = eorder[np.searchsorted(ekey, k, sorter=eorder)]
                np.bitwise_or.at(tag, P + pos, ftag)
    return dict(dim=3, xyz=xyz, conn=conn, tag=tag, n_vertices=P,
                name=f"bifurcation h={h} Lp={parent_len} s={stenosis} Rd={daughter_radius} Ld={L_d}",
                radius=radius, length=parent_len, stenosis=stenosis)
