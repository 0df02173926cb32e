"""Graph aggregates of the coarse Schur correction (host code of the library,
called through the C ABI; no GPU needed): exact partitions of path graphs,
and on the vertex graphs of the benchmark-family pipes the properties the
correction relies on (a partition, connected aggregates, none crossing a
component, bounded counts, numbering by component)."""

import numpy as np
import pytest

from paper_2009_06725_gb300 import scvs
from synthetic import workloads


def csr_from_edges(n, edges):
    nb = [set() for _ in range(n)]
    for a, b in edges:
        nb[a].add(b)
        nb[b].add(a)
    ptr = np.zeros(n + 1, dtype=np.int64)
    col = []
    for v in range(n):
        row = sorted(nb[v] | {v})
        col += row
        ptr[v + 1] = ptr[v] + len(row)
    return ptr, np.array(col, dtype=np.int32)


def path(n):
    return csr_from_edges(n, [(i, i + 1) for i in range(n - 1)])


def vertex_graph(mesh):
    """P1 adjacency of the mesh's vertices (the vertices of every element are pairwise adjacent)."""
    P = mesh["n_vertices"]
    nv = mesh["dim"] + 1
    cv = mesh["conn"][:, :nv].astype(np.int64)
    assert cv.max() < P
    rows = np.repeat(cv, nv, axis=1).ravel()
    cols = np.tile(cv, (1, nv)).ravel()
    key = np.unique(rows * P + cols)
    r, c = key // P, key % P
    ptr = np.zeros(P + 1, dtype=np.int64)
    np.add.at(ptr, r + 1, 1)
    return np.cumsum(ptr), c.astype(np.int32)


def components(ptr, col):
    n = ptr.size - 1
    comp = -np.ones(n, dtype=np.int64)
    k = 0
    for s in range(n):
        if comp[s] >= 0:
            continue
        comp[s] = k
        stack = [s]
        while stack:
            v = stack.pop()
            for u in col[ptr[v]:ptr[v + 1]]:
                if comp[u] < 0:
                    comp[u] = k
                    stack.append(u)
        k += 1
    return comp, k


def check_partition(ptr, col, agg, n_agg, n_blk, target):
    n = ptr.size - 1
    comp, k = components(ptr, col)
    assert n_blk == k
    assert agg.min() == 0 and agg.max() == n_agg - 1 and np.unique(agg).size == n_agg
    # each aggregate in one component, and connected
    for a in range(n_agg):
        vs = np.flatnonzero(agg == a)
        assert np.unique(comp[vs]).size == 1
        seen = {int(vs[0])}
        stack = [int(vs[0])]
        inside = set(vs.tolist())
        while stack:
            v = stack.pop()
            for u in col[ptr[v]:ptr[v + 1]]:
                u = int(u)
                if u in inside and u not in seen:
                    seen.add(u)
                    stack.append(u)
        assert len(seen) == vs.size, a
    # numbering: by component (in order of the lowest vertex), contiguous
    blk_of_agg = np.array([comp[np.flatnonzero(agg == a)[0]] for a in range(n_agg)])
    assert np.all(np.diff(blk_of_agg) >= 0)
    counts = np.bincount(blk_of_agg, minlength=k)
    assert counts.max() <= min(2 * target, 1024)
    return comp, counts


@pytest.mark.parametrize("n,target,expect", [
    (10, 2, [5, 5]),          # cap ceil(10/2) = 5
    (10, 3, [4, 4, 2]),       # cap 4, remainder 2 is not below a third of 4
    (10, 5, [2] * 5),
    (13, 4, [4, 4, 5]),       # cap 4: remainder {12} (size 1 < 4/3) joins its neighbour's aggregate
    (7, 20, [1] * 7),         # fewer vertices than the target: one vertex each
])
def test_path_graph_exact(n, target, expect):
    ptr, col = path(n)
    agg, n_agg, n_blk = scvs.scvs_graph_aggregates(ptr, col, target)
    assert n_blk == 1 and n_agg == len(expect)
    assert np.bincount(agg).tolist() == expect
    assert np.all(np.diff(agg) >= 0)  # breadth-first growth along a path keeps runs


def test_interleaved_components_numbered_by_component():
    # component A: even vertices in a path, component B: odd vertices in a path
    n = 20
    edges = [(i, i + 2) for i in range(0, n - 2)]
    ptr, col = csr_from_edges(n, edges)
    agg, n_agg, n_blk = scvs.scvs_graph_aggregates(ptr, col, 2)
    assert n_blk == 2 and n_agg == 4
    assert set(agg[0::2].tolist()) == {0, 1} and set(agg[1::2].tolist()) == {2, 3}
    check_partition(ptr, col, agg, n_agg, n_blk, 2)


def test_long_pipe_vertex_graph():
    # L/R = 40 pipe of the batch family: the elongated case the correction targets
    wl = workloads.pipe_workload(n_c=3, n_r=2, n_x=120, n_modes=1, length=40.0, radius=1.0)
    ptr, col = vertex_graph(wl["mesh"])
    for target in (24, 96):
        agg, n_agg, n_blk = scvs.scvs_graph_aggregates(ptr, col, target)
        _, counts = check_partition(ptr, col, agg, n_agg, n_blk, target)
        assert n_blk == 1
        assert target // 2 <= counts[0] <= 2 * target
        # the aggregates tile the pipe's length: their mean axial positions spread over [0, L]
        x = wl["mesh"]["xyz"][:ptr.size - 1, 0]
        xm = np.array([x[agg == a].mean() for a in range(n_agg)])
        assert xm.min() < 40.0 / n_agg * 4 and xm.max() > 40.0 - 40.0 / n_agg * 4
        again = scvs.scvs_graph_aggregates(ptr, col, target)[0]
        assert np.array_equal(agg, again)


def test_union_of_uneven_pipes():
    wls = workloads.uneven_pipes(n_meshes=3, n_modes=2, seed=3, n_min=2000, n_max=20000)
    u = workloads.union_workload(wls)
    ptr, col = vertex_graph(u["mesh"])
    agg, n_agg, n_blk = scvs.scvs_graph_aggregates(ptr, col, 32)
    comp, counts = check_partition(ptr, col, agg, n_agg, n_blk, 32)
    assert n_blk == 3
    # the graph components are the union's meshes
    node_comp = np.asarray(u["node_comp"])[:ptr.size - 1]
    for b in range(3):
        assert np.unique(node_comp[comp == b]).size == 1
    assert np.all(counts >= 8)


def test_bad_arguments():
    ptr, col = path(5)
    with pytest.raises(scvs.ScvsError):
        scvs.scvs_graph_aggregates(ptr, col, 0)
    with pytest.raises(scvs.ScvsError):
        scvs.scvs_graph_aggregates(ptr, col, 513)
    bad = col.copy()
    bad[3] = 5
    with pytest.raises(scvs.ScvsError):
        scvs.scvs_graph_aggregates(ptr, bad, 2)
    agg, n_agg, n_blk = scvs.scvs_graph_aggregates(np.zeros(1, dtype=np.int64), np.zeros(0, dtype=np.int32), 4)
    assert agg.size == 0 and n_agg == 0 and n_blk == 0


def test_default_aggregate_count():
    o = scvs.scvs_default_opts()
    assert o.schur_agg == 16 and o.precond == scvs.SCVS_PC_AUTO


def _random_graph(n, n_comp, extra, seed):
    """n vertices in n_comp components: a random spanning tree per component plus
    extra random edges inside components; vertex ids shuffled across components."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n)
    parts = np.array_split(perm, n_comp)
    edges = []
    for part in parts:
        for i in range(1, part.size):
            edges.append((int(part[i]), int(part[rng.integers(0, i)])))
        for _ in range(extra if part.size > 1 else 0):
            a, b = rng.choice(part, 2, replace=False)
            edges.append((int(a), int(b)))
    return csr_from_edges(n, edges)


def test_random_graphs_property():
    hypothesis = pytest.importorskip("hypothesis")
    st = hypothesis.strategies

    @hypothesis.settings(max_examples=40, deadline=None)
    @hypothesis.given(n=st.integers(1, 300), n_comp=st.integers(1, 6), extra=st.integers(0, 200),
                      target=st.integers(1, 64), seed=st.integers(0, 2**31 - 1))
    def prop(n, n_comp, extra, target, seed):
        n_comp = min(n_comp, n)
        ptr, col = _random_graph(n, n_comp, extra, seed)
        agg, n_agg, n_blk = scvs.scvs_graph_aggregates(ptr, col, target)
        assert n_blk == n_comp
        check_partition(ptr, col, agg, n_agg, n_blk, target)
        assert np.array_equal(agg, scvs.scvs_graph_aggregates(ptr, col, target)[0])

    prop()
