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
           stenosis=0.0, core=0.5):
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
    vertex/edge counts.
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
