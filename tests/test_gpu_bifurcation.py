"""The stenosed bifurcation (voxel mesh of the parent, junction and two
daughters) through the C ABI: patterns bit-exact and values against the
oracle's assembly; FP64 and mixed solves against the oracle's LU on a small
instance (whose LU the oracle finishes in seconds); and, on a mid-size
instance beyond the oracle's reach, the mixed path against the FP64 path with
the oracle's residual definition checked on sampled modes."""
import numpy as np
import pytest

from oracle import fem
from paper_2009_06725_gb300 import scvs
from synthetic import workloads

from .gpu_util import rel_err, rel_l2, solve, stack_modal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small():
    wl = workloads.bifurcation_workload(h=0.4, n_modes=4)
    mats = fem.assemble(wl["mesh"])
    return wl, mats, fem.solve_modes(mats, wl)


def test_patterns_and_values(small):
    wl, mats, _ = small
    s = scvs.Solver()
    with s:
        mid = scvs.scvs_set_mesh(s.ctx, wl["mesh"])
        pat = fem.patterns(mats["N"], mats["P"], wl["mesh"]["conn"], 3)
        for which, key in ((scvs.SCVS_CSR_S, "S"), (scvs.SCVS_CSR_G, "G"), (scvs.SCVS_CSR_GT, "GT")):
            rp, col = scvs.scvs_get_csr(s.ctx, mid, which)
            assert np.array_equal(rp, pat[key][0]) and np.array_equal(col, pat[key][1]), key
        v = scvs.scvs_get_values(s.ctx, mid, scvs.SCVS_CSR_S, 3)
        assert rel_err(v[0], mats["Ms"].data) < 1e-12 and rel_err(v[1], mats["Ks"].data) < 1e-12
        v = scvs.scvs_get_values(s.ctx, mid, scvs.SCVS_CSR_G, 3)
        for c in range(3):
            assert rel_err(v[c], mats["D"][c].data) < 1e-12


@pytest.mark.parametrize("precision,solve_tol,err_tol", [(scvs.SCVS_PREC_FP64, 1e-13, 1e-10),
                                                         (scvs.SCVS_PREC_MIXED, 1e-12, 1e-8)])
def test_solve_matches_oracle(small, precision, solve_tol, err_tol):
    wl, mats, X = small
    s, mid, rep, u, p = solve(wl, precision=precision, tol=solve_tol, restart=20, max_cycles=2000)
    with s:
        Xg = stack_modal(u, p)
    for k, r in enumerate(rep):
        assert r["status"] == scvs.SCVS_CONVERGED, (k, r)
        assert rel_l2(Xg[k], X[k]) < err_tol, (k, rel_l2(Xg[k], X[k]))
    assert np.all(fem.relative_residual(mats, wl, Xg) < 10 * solve_tol)


def test_mixed_matches_fp64_mid_size():
    wl = workloads.bifurcation_workload(h=0.15, n_modes=16)
    res = {}
    for precision in (scvs.SCVS_PREC_FP64, scvs.SCVS_PREC_MIXED):
        s, mid, rep, u, p = solve(wl, precision=precision, tol=1e-12, restart=20, max_cycles=2000)
        s.close()
        assert all(r["status"] == scvs.SCVS_CONVERGED for r in rep), rep
        res[precision] = stack_modal(u, p)
    A, B = res[scvs.SCVS_PREC_FP64], res[scvs.SCVS_PREC_MIXED]
    for k in range(16):
        assert rel_l2(B[k], A[k]) < 1e-8, (k, rel_l2(B[k], A[k]))
    mats = fem.assemble(wl["mesh"])
    sample = [0, 5, 15]
    sub = dict(wl, omegas=wl["omegas"][sample], g=wl["g"][sample])
    assert np.all(fem.relative_residual(mats, sub, B[sample]) < 1e-11)
