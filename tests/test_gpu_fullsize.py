"""Parity at the benchmark's full size (151k-node pipe, 32 modes) in the
configuration bench.py times: complete pattern and value comparison,
operator on sampled modes, and the converged solve checked by the oracle's
own residual definition on sampled modes and against the analytic
Womersley flow (a property that holds at any size)."""
import numpy as np
import pytest

from oracle import fem
from paper_2009_06725_gb300 import scvs
from synthetic import workloads

from .gpu_util import apply_gpu, rel_err, stack_modal

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def full():
    wl = workloads.pipe_workload()  # the benchmark pipe
    mats = fem.assemble(wl["mesh"])
    s = scvs.Solver()
    mid = scvs.scvs_set_mesh(s.ctx, wl["mesh"])
    scvs.scvs_set_physics(s.ctx, mid, wl["rho"], wl["mu"])
    scvs.scvs_set_modes(s.ctx, mid, wl["omegas"], wl["g"])
    yield wl, mats, s, mid
    s.close()


def test_full_patterns_and_values(full):
    wl, mats, s, mid = full
    pat = fem.patterns(mats["N"], mats["P"], wl["mesh"]["conn"], 3)
    for which, key in ((scvs.SCVS_CSR_S, "S"), (scvs.SCVS_CSR_G, "G"), (scvs.SCVS_CSR_GT, "GT")):
        rp, col = scvs.scvs_get_csr(s.ctx, mid, which)
        assert np.array_equal(rp, pat[key][0]) and np.array_equal(col, pat[key][1]), key
    v = scvs.scvs_get_values(s.ctx, mid, scvs.SCVS_CSR_S, 3)
    assert rel_err(v[0], mats["Ms"].data) < 1e-12 and rel_err(v[1], mats["Ks"].data) < 1e-12
    v = scvs.scvs_get_values(s.ctx, mid, scvs.SCVS_CSR_G, 3)
    for c in range(3):
        assert rel_err(v[c], mats["D"][c].data) < 1e-12


def test_full_operator_sampled_modes(full):
    wl, mats, s, mid = full
    n = fem.dof_count(mats)
    X = workloads.random_block(n, 32, seed=5)
    Yg64 = apply_gpu(s, mid, X, scvs.SCVS_PREC_FP64)
    Yg32 = apply_gpu(s, mid, X, scvs.SCVS_PREC_MIXED)
    for k in (0, 13, 31):
        Y = fem.masked_apply(mats, wl["omegas"][k:k + 1], wl["rho"], wl["mu"], wl["dir_nodes"], X[:, k:k + 1])[:, 0]
        assert rel_err(Yg64[:, k], Y) < 1e-12
        assert rel_err(Yg32[:, k], Y) < 1e-5


def test_full_solve_converges_to_oracle_residual(full):
    wl, mats, s, mid = full
    rep = scvs.scvs_solve(s.ctx, mid, 32)
    assert all(r["status"] == scvs.SCVS_CONVERGED and r["rel_res"] <= 1e-8 for r in rep)
    u, p = scvs.scvs_get_modal(s.ctx, mid, 32, mats["N"], 3, mats["P"])
    X = stack_modal(u, p)
    sample = [0, 7, 19, 31]
    sub = dict(wl, omegas=wl["omegas"][sample], g=wl["g"][sample])
    rr = fem.relative_residual(mats, sub, X[sample])
    assert np.all(rr < 1.05e-8), rr
    for k in range(32):  # polygonal pipe: close to the continuum Womersley flow
        ue, _ = workloads.exact_nodal(wl, k)
        assert fem.relative_l2_error(mats["Ms"], ue, u[k]) < 2e-2
