"""Invariants of the seeded inputs that are not covered elsewhere: the union
mesh of a batch (vertex-first numbering, components disjoint, data carried
over exactly) and the uneven stenosed-pipe batch (sizes, ranges, seeding).
These generators carry no method arithmetic; they are the shared inputs of
the oracle and the CUDA path."""
import numpy as np

from synthetic import meshes, workloads


def _small_batch():
    return [workloads.pipe_workload(n_c=2 + i, n_r=1 + i % 2, n_x=3 + i, n_modes=3, length=2.0 + i,
                                    radius=0.6 + 0.2 * i, stenosis=0.1 * i, seed=i) for i in range(3)]


def test_union_mesh_is_a_disjoint_vertex_first_union():
    parts = _small_batch()
    U = workloads.union_workload(parts)
    mesh, comp, maps = U["mesh"], U["node_comp"], U["maps"]
    P = mesh["n_vertices"]
    assert P == sum(p["mesh"]["n_vertices"] for p in parts)
    assert mesh["xyz"].shape[0] == sum(p["mesh"]["xyz"].shape[0] for p in parts)
    for i, (p, mp) in enumerate(zip(parts, maps)):
        m = p["mesh"]
        Pi = m["n_vertices"]
        # vertices of every component among the union's vertices, edge nodes after them
        assert np.all(mp[:Pi] < P) and np.all(mp[Pi:] >= P)
        assert np.array_equal(mesh["xyz"][mp], m["xyz"]) and np.array_equal(mesh["tag"][mp], m["tag"])
        assert np.all(comp[mp] == i)
    # the map is a bijection onto the union's nodes
    allmap = np.concatenate(maps)
    assert np.array_equal(np.sort(allmap), np.arange(mesh["xyz"].shape[0]))
    # no element couples two components
    ec = comp[mesh["conn"]]
    assert np.all(ec == ec[:, :1])
    # Dirichlet data land on the union's Dirichlet nodes of the right component
    pos = {int(n): j for j, n in enumerate(U["dir_nodes"])}
    for p, mp in zip(parts, maps):
        idx = [pos[int(mp[n])] for n in p["dir_nodes"]]
        assert np.array_equal(U["g"][:, idx, :], p["g"])


def test_uneven_pipes_sizes_and_seeding():
    a = workloads.uneven_pipes(n_meshes=6, n_modes=4, seed=3, scale=0.05)
    b = workloads.uneven_pipes(n_meshes=6, n_modes=4, seed=3, scale=0.05)
    for wa, wb in zip(a, b):  # seeded: identical on every call
        assert np.array_equal(wa["mesh"]["xyz"], wb["mesh"]["xyz"]) and np.array_equal(wa["g"], wb["g"])
    for w in a:
        m = w["mesh"]
        assert 0.5 <= m["radius"] <= 1.5 and 5.0 <= m["length"] <= 20.0 and 0.0 <= m["stenosis"] <= 0.5
        assert m["xyz"].shape[0] >= 0.05 * 20_000 / 4   # within a factor of the log-uniform target range
        assert (m["tag"] & meshes.OUTLET).any() and (m["tag"] & meshes.INLET).any()
        # |c_k| = k^-2 for k >= 1, c_0 = 1
        c = w["coeffs"]
        assert abs(c[0] - 1) < 1e-15 and np.allclose(np.abs(c[1:]), np.arange(1, 4) ** -2.0)
