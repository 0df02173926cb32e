"""Many meshes of uneven size in one solve: a union mesh of independent
components, every (component, mode) its own system, against the oracle's
per-mesh solves."""
import numpy as np
import pytest

from oracle import fem
from paper_2009_06725_gb300 import scvs
from synthetic import meshes, workloads

pytestmark = pytest.mark.gpu


def _parts():
    sizes = [(2, 1, 3, 1.5, 0.7), (3, 2, 5, 2.5, 1.2), (2, 2, 4, 2.0, 1.0)]
    wls = []
    for i, (n_c, n_r, n_x, L, R) in enumerate(sizes):
        wl = workloads.pipe_workload(n_c=n_c, n_r=n_r, n_x=n_x, n_modes=5, length=L, radius=R,
                                     stenosis=0.2 * i, seed=i)
        wls.append(wl)
    return wls


@pytest.mark.parametrize("precision", [scvs.SCVS_PREC_MIXED, scvs.SCVS_PREC_FP64])
def test_batched_components_match_per_mesh_oracle(precision):
    wls = _parts()
    U = workloads.union_workload(wls)
    m = len(U["omegas"])
    tol = 1e-12 if precision == scvs.SCVS_PREC_MIXED else 1e-13
    with scvs.Solver(precision=precision, tol=tol, max_cycles=2000) as s:
        mid = scvs.scvs_set_mesh(s.ctx, U["mesh"])
        scvs.scvs_set_components(s.ctx, mid, U["n_comp"], U["node_comp"])
        scvs.scvs_set_physics(s.ctx, mid, U["rho"], U["mu"])
        scvs.scvs_set_modes(s.ctx, mid, U["omegas"], U["g"])
        rep = scvs.scvs_solve(s.ctx, mid, U["n_comp"] * m)
        N, P = U["mesh"]["xyz"].shape[0], U["mesh"]["n_vertices"]
        u, p = scvs.scvs_get_modal(s.ctx, mid, m, N, 3, P)
    assert len(rep) == 3 * m
    for i, (wl, mp) in enumerate(zip(wls, U["maps"])):
        mats = fem.assemble(wl["mesh"])
        X = fem.solve_modes(mats, wl)
        Pi = wl["mesh"]["n_vertices"]
        for k in range(m):
            r = rep[i * m + k]
            assert r["status"] == scvs.SCVS_CONVERGED, (i, k, r)
            xi = np.concatenate([u[k][mp].reshape(-1), p[k][mp[:Pi]]])
            err = np.linalg.norm(xi - X[k]) / np.linalg.norm(X[k])
            assert err < (1e-8 if precision == scvs.SCVS_PREC_MIXED else 1e-10), (i, k, err)


def test_components_are_independent_systems():
    """Scaling one component's data by 1e6 changes nothing in the others'
    iteration counts or solutions (no shared Krylov space)."""
    wls = _parts()
    U1 = workloads.union_workload(wls)
    big = dict(wls[1], g=wls[1]["g"] * 1e6)
    U2 = workloads.union_workload([wls[0], big, wls[2]])
    m = len(U1["omegas"])
    out = []
    for U in (U1, U2):
        with scvs.Solver() as s:
            mid = scvs.scvs_set_mesh(s.ctx, U["mesh"])
            scvs.scvs_set_components(s.ctx, mid, U["n_comp"], U["node_comp"])
            scvs.scvs_set_physics(s.ctx, mid, U["rho"], U["mu"])
            scvs.scvs_set_modes(s.ctx, mid, U["omegas"], U["g"])
            rep = scvs.scvs_solve(s.ctx, mid, U["n_comp"] * m)
            N, P = U["mesh"]["xyz"].shape[0], U["mesh"]["n_vertices"]
            u, p = scvs.scvs_get_modal(s.ctx, mid, m, N, 3, P)
        out.append((rep, u))
    for i in (0, 2):
        for k in range(m):
            assert out[0][0][i * m + k]["iterations"] == out[1][0][i * m + k]["iterations"]
            mp = U1["maps"][i]
            assert np.array_equal(out[0][1][k][mp], out[1][1][k][mp])


def test_components_rejected_when_coupled():
    m = meshes.pipe3d(n_c=2, n_r=1, n_x=2)
    nc = np.zeros(m["xyz"].shape[0], dtype=np.int32)
    nc[5] = 1
    with scvs.Solver() as s:
        mid = scvs.scvs_set_mesh(s.ctx, m)
        with pytest.raises(scvs.ScvsError) as e:
            scvs.scvs_set_components(s.ctx, mid, 2, nc)
        assert e.value.code == scvs.SCVS_ERR_MESH
