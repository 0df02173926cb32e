"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars: patterns and indexing bit-exact; FP64 values and FP64 operator within
1e-12 (max-abs relative); FP32 operator within 1e-5; FP64 solve within 1e-10
and mixed-precision solve within 1e-8 relative L2 per mode (solved to
1e-13 / 1e-12 residual so that the residual does not dominate the error).
"""
import numpy as np
import pytest

from oracle import fem
from paper_2009_06725_gb300 import scvs
from synthetic import meshes, workloads

from .gpu_util import apply_gpu, open_workload, rel_err, rel_l2, solve, stack_modal

pytestmark = pytest.mark.gpu

CASES = {
    "channel32x8": lambda: workloads.channel_workload(32, 8, n_modes=8),
    "pipe_small": lambda: workloads.pipe_workload(n_c=3, n_r=2, n_x=6, n_modes=5, length=2.0),
    "channel_tiny": lambda: workloads.channel_workload(2, 1, n_modes=3),
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    wl = CASES[request.param]()
    mats = fem.assemble(wl["mesh"])
    return request.param, wl, mats


def test_patterns_bit_exact(case):
    _, wl, mats = case
    m = wl["mesh"]
    pat = fem.patterns(mats["N"], mats["P"], m["conn"], m["dim"])
    s, mid = open_workload(wl)
    with s:
        for which, key in ((scvs.SCVS_CSR_S, "S"), (scvs.SCVS_CSR_G, "G"), (scvs.SCVS_CSR_GT, "GT")):
            rp, col = scvs.scvs_get_csr(s.ctx, mid, which)
            assert np.array_equal(rp, pat[key][0]), key
            assert np.array_equal(col, pat[key][1]), key
        # Q (P1 x P1) = vertex rows restricted to vertex columns
        rp, col = scvs.scvs_get_csr(s.ctx, mid, scvs.SCVS_CSR_Q)
        gp, gc = pat["G"]
        P = mats["P"]
        assert np.array_equal(rp, gp[: P + 1]) and np.array_equal(col, gc[: gp[P]])


def test_values_match_oracle(case):
    _, wl, mats = case
    s, mid = open_workload(wl)
    d = wl["mesh"]["dim"]
    with s:
        v = scvs.scvs_get_values(s.ctx, mid, scvs.SCVS_CSR_S, d)
        assert rel_err(v[0], mats["Ms"].data) < 1e-12
        assert rel_err(v[1], mats["Ks"].data) < 1e-12
        v = scvs.scvs_get_values(s.ctx, mid, scvs.SCVS_CSR_G, d)
        for c in range(d):
            assert rel_err(v[c], mats["D"][c].data) < 1e-12
        v = scvs.scvs_get_values(s.ctx, mid, scvs.SCVS_CSR_GT, d)
        for c in range(d):
            DT = mats["D"][c].T.tocsr()
            DT.sort_indices()
            assert rel_err(v[c], DT.data) < 1e-12
        v = scvs.scvs_get_values(s.ctx, mid, scvs.SCVS_CSR_Q, d)
        Mp, Lp = fem.p1_diagonals(wl["mesh"])
        rp, col = scvs.scvs_get_csr(s.ctx, mid, scvs.SCVS_CSR_Q)
        diag = np.array([v[0][rp[i]:rp[i + 1]][col[rp[i]:rp[i + 1]] == i][0] for i in range(mats["P"])])
        assert rel_err(diag, Mp) < 1e-12
        diagl = np.array([v[1][rp[i]:rp[i + 1]][col[rp[i]:rp[i + 1]] == i][0] for i in range(mats["P"])])
        assert rel_err(diagl, Lp) < 1e-12
        # P1 mass row sums = int N_B (sums to the volume)
        assert np.isclose(v[0].sum(), np.ones(mats["N"]) @ mats["Ms"] @ np.ones(mats["N"]), rtol=1e-12)


@pytest.mark.parametrize("precision,tol", [(scvs.SCVS_PREC_FP64, 1e-12), (scvs.SCVS_PREC_MIXED, 1e-5)])
@pytest.mark.parametrize("matfree", [False, True])
def test_operator_matches_oracle(case, precision, tol, matfree):
    _, wl, mats = case
    n = fem.dof_count(mats)
    m = len(wl["omegas"])
    X = workloads.random_block(n, m, seed=11)
    Y = fem.masked_apply(mats, wl["omegas"], wl["rho"], wl["mu"], wl["dir_nodes"], X)
    s, mid = open_workload(wl)
    with s:
        Yg = apply_gpu(s, mid, X, precision, matfree=matfree)
    for k in range(m):
        assert rel_err(Yg[:, k], Y[:, k]) < tol, (k, rel_err(Yg[:, k], Y[:, k]))


def test_rhs_lift_matches_oracle(case):
    _, wl, mats = case
    B = fem.rhs_block(mats, wl)
    s, mid = open_workload(wl)
    with s:
        ptr = scvs.scvs_rhs_dev(s.ctx, mid)
        ld = scvs.scvs_mode_stride(s.ctx, mid)
        n = fem.dof_count(mats)
        Bg = _device_view(ptr, n * ld).reshape(n, ld)
    for k in range(len(wl["omegas"])):
        assert rel_err(Bg[:, k], B[:, k]) < 1e-12


def _device_view(ptr, count):
    """Copy `count` complex128 values at device address ptr to the host
    (zero-copy torch view through the CUDA array interface, then .cpu())."""
    import torch

    class _View:
        __cuda_array_interface__ = {"shape": (count,), "typestr": "<c16", "data": (ptr, False), "version": 3}

    return torch.as_tensor(_View(), device="cuda").cpu().numpy()


@pytest.mark.parametrize("precision,solve_tol,err_tol", [(scvs.SCVS_PREC_FP64, 1e-13, 1e-10),
                                                         (scvs.SCVS_PREC_MIXED, 1e-12, 1e-8)])
def test_solve_matches_oracle(case, precision, solve_tol, err_tol):
    name, wl, mats = case
    X = fem.solve_modes(mats, wl)
    s, mid, rep, u, p = solve(wl, precision=precision, tol=solve_tol, max_cycles=2000)
    with s:
        Xg = stack_modal(u, p)
    for k, r in enumerate(rep):
        assert r["status"] == scvs.SCVS_CONVERGED, (k, r)
        assert r["rel_res"] <= solve_tol
        assert rel_l2(Xg[k], X[k]) < err_tol, (k, rel_l2(Xg[k], X[k]))
    # the library's residual agrees with the oracle's definition
    rr = fem.relative_residual(mats, wl, Xg)
    assert np.all(rr < 10 * solve_tol)


def test_reconstruction_matches_oracle():
    wl = workloads.channel_workload(32, 8, n_modes=8)
    mats = fem.assemble(wl["mesh"])
    s, mid, rep, u, p = solve(wl, precision=scvs.SCVS_PREC_FP64, tol=1e-12)
    n_t = 24
    with s:
        ut, pt = scvs.scvs_reconstruct(s.ctx, mid, n_t, wl["period"], mats["N"], 2, mats["P"])
    ref_u = fem.reconstruct(u, wl["omegas"], n_t, wl["period"])
    ref_p = fem.reconstruct(p, wl["omegas"], n_t, wl["period"])
    assert rel_err(ut, ref_u) < 1e-12
    assert rel_err(pt, ref_p) < 1e-12


def test_channel_mode0_poiseuille_on_gpu():
    wl = workloads.channel_workload(32, 8, n_modes=1)
    s, mid, rep, u, p = solve(wl, precision=scvs.SCVS_PREC_FP64, tol=1e-13)
    s.close()
    ue, pe = workloads.exact_nodal(wl, 0)
    assert np.abs(u[0] - ue).max() < 1e-9 * np.abs(ue).max()
    assert np.abs(p[0] - pe).max() < 1e-8 * np.abs(pe).max()


def test_mode_counts_and_padding():
    """n_modes that are not powers of two (padding columns) and one mode."""
    for nm in (1, 3, 5):
        wl = workloads.pipe_workload(n_c=2, n_r=1, n_x=3, n_modes=nm, length=1.5)
        mats = fem.assemble(wl["mesh"])
        X = fem.solve_modes(mats, wl)
        s, mid, rep, u, p = solve(wl, tol=1e-12)
        s.close()
        Xg = stack_modal(u, p)
        for k in range(nm):
            assert rep[k]["status"] == scvs.SCVS_CONVERGED
            assert rel_l2(Xg[k], X[k]) < 1e-8


def test_zero_data_mode_and_nonfinite_isolation():
    wl = workloads.pipe_workload(n_c=2, n_r=1, n_x=3, n_modes=4, length=1.5)
    g = wl["g"].copy()
    g[1] = 0.0                      # zero data: exact answer x = 0
    g[2, 0, 0] = np.nan             # non-finite data in mode 2 only
    wl2 = dict(wl, g=g)
    mats = fem.assemble(wl["mesh"])
    X = fem.solve_modes(mats, dict(wl, g=np.where(np.isnan(g), 0, g)))
    s, mid, rep, u, p = solve(wl2, tol=1e-12)
    s.close()
    Xg = stack_modal(u, p)
    assert rep[1]["status"] == scvs.SCVS_CONVERGED and np.abs(Xg[1]).max() == 0.0
    assert rep[2]["status"] == scvs.SCVS_NON_FINITE
    for k in (0, 3):
        assert rep[k]["status"] == scvs.SCVS_CONVERGED
        assert rel_l2(Xg[k], X[k]) < 1e-8


def test_cycle_cap_reports_max_iter():
    wl = workloads.pipe_workload(n_c=3, n_r=2, n_x=6, n_modes=2, length=2.0)
    s, mid, rep, u, p = solve(wl, max_cycles=1, restart=2, cheb_u=1, cheb_m=1, cheb_l=1)
    s.close()
    assert all(r["status"] == scvs.SCVS_MAX_ITER for r in rep)
    assert all(r["rel_res"] > 1e-8 for r in rep)


def test_invalid_meshes_rejected():
    m = meshes.channel2d(2, 1)
    s = scvs.Solver()
    with s:
        bad = dict(m, conn=m["conn"].copy())
        bad["conn"][0, [1, 2]] = bad["conn"][0, [2, 1]]  # inverted triangle
        with pytest.raises(scvs.ScvsError) as e:
            scvs.scvs_set_mesh(s.ctx, bad)
        assert e.value.code == scvs.SCVS_ERR_MESH
        bad = dict(m, conn=m["conn"].copy())
        bad["conn"][1, 4] = m["xyz"].shape[0] + 5  # out of range
        with pytest.raises(scvs.ScvsError) as e:
            scvs.scvs_set_mesh(s.ctx, bad)
        assert e.value.code == scvs.SCVS_ERR_MESH
        t = m["tag"]
        closed = dict(m, tag=np.where(t & 4, (t & np.uint8(0xFB)) | np.uint8(1), t).astype(np.uint8))
        with pytest.raises(scvs.ScvsError) as e:
            scvs.scvs_set_mesh(s.ctx, closed)
        assert e.value.code == scvs.SCVS_ERR_PRESSURE_NULLSPACE
        # the context stays usable after the errors
        mid = scvs.scvs_set_mesh(s.ctx, m)
        assert mid == 0
