"""Staged gathers (row blocks with the footprint copied into shared memory by
TMA bulk copies) against their definition and against the unstaged kernels.

* The row blocks: perm is a permutation of the nodes, the blocks cover it in
  order, each footprint is exactly the sorted set of distinct columns of its
  block's rows (recomputed here from the S pattern), its vertex prefix is the
  count of columns below n_vertices, and every nonzero's local index points
  at its own column.
* The staged FP32 SpMM and preconditioner visit every row's nonzeros in the
  same order with the same arithmetic as the unstaged kernels, so their
  outputs are identical, for every mode chunk and in 2D and 3D.
* Solves with staging forced reach the oracle's solutions at the parity
  tolerance."""
import numpy as np
import pytest

from oracle import fem
from paper_2009_06725_gb300 import scvs
from synthetic import workloads

from .gpu_util import open_workload, padded_block, rel_l2, solve, stack_modal, torch_cuda

pytestmark = pytest.mark.gpu


def _cases():
    return {
        "pipe": workloads.pipe_workload(n_c=3, n_r=2, n_x=10, n_modes=32, length=5.0),
        "channel": workloads.channel_workload(32, 8, n_modes=8),
    }


@pytest.fixture(scope="module", params=["pipe", "channel"])
def case(request):
    return request.param, _cases()[request.param]


def test_row_blocks_match_their_definition(case):
    name, wl = case
    mesh = wl["mesh"]
    N, P = mesh["xyz"].shape[0], mesh["n_vertices"]
    s, mid = open_workload(wl, stage=0)
    with s:
        info = scvs.scvs_staged_info(s.ctx, mid)
        assert info["valid"] and info["n_blk"] >= 2
        ptr, col = scvs.scvs_get_csr(s.ctx, mid, scvs.SCVS_CSR_S)
        rb = scvs.scvs_staged_blocks(s.ctx, mid, N, col.size)
    perm, row0, fp_ptr, fp_col, fv_len, lcol = (rb[k] for k in ("perm", "row0", "fp_ptr", "fp_col", "fv_len", "lcol"))
    assert np.array_equal(np.sort(perm), np.arange(N))
    assert row0[0] == 0 and row0[-1] == N and np.all(np.diff(row0) > 0)
    assert fp_ptr[0] == 0 and fp_ptr[-1] == fp_col.size == info["fp_total"]
    lens = np.diff(ptr)
    for b in range(info["n_blk"]):
        rows = perm[row0[b]:row0[b + 1]]
        cols = np.concatenate([col[ptr[r]:ptr[r + 1]] for r in rows])
        assert cols.size <= info["budget"] + lens.max()
        fp = fp_col[fp_ptr[b]:fp_ptr[b + 1]]
        assert np.array_equal(fp, np.unique(cols))
        assert fv_len[b] == int((fp < P).sum())
        for r in rows:
            assert np.array_equal(fp[lcol[ptr[r]:ptr[r + 1]]], col[ptr[r]:ptr[r + 1]])
    assert info["fp_max"] == int(np.diff(fp_ptr).max()) and info["fv_max"] == int(fv_len.max())
    # blocks are compact: every block needs far fewer distinct columns than nonzeros
    assert fp_col.size < 0.6 * col.size


def _run(wl, stage, X, R):
    """SpMM and preconditioner of one context with the given stage option."""
    torch = torch_cuda()
    s, mid = open_workload(wl, stage=stage)
    with s:
        ld = scvs.scvs_mode_stride(s.ctx, mid)
        info = scvs.scvs_staged_info(s.ctx, mid)
        x = torch.from_numpy(padded_block(X, ld)).to(torch.complex64).cuda()
        r = torch.from_numpy(padded_block(R, ld)).to(torch.complex64).cuda()
        y, z = torch.zeros_like(x), torch.zeros_like(r)
        torch.cuda.synchronize()
        scvs.scvs_apply(s.ctx, mid, scvs.SCVS_PREC_MIXED, x.data_ptr(), y.data_ptr())
        scvs.scvs_apply_precond(s.ctx, mid, r.data_ptr(), z.data_ptr())
        torch.cuda.synchronize()
        return info, y.cpu().numpy(), z.cpu().numpy()


def test_staged_kernels_equal_unstaged(case):
    name, wl = case
    m = len(wl["omegas"])
    mats = fem.assemble(wl["mesh"])
    n = fem.dof_count(mats)
    X = workloads.random_block(n, m, seed=5)
    R = workloads.random_block(n, m, seed=6)
    info0, y0, z0 = _run(wl, -1, X, R)
    assert not info0["valid"] and info0["st_spmm"] == 0 and info0["st_cheb"] == 0
    ld = y0.shape[1]
    for mc in (4, 8, 16, 32):
        if mc > ld:
            continue
        info, y, z = _run(wl, mc, X, R)
        assert info["st_spmm"] == mc and info["st_cheb"] == mc
        if mc <= 16:  # the small footprints of these meshes fit shared memory up to 16 modes per block
            assert info["runs_spmm"] and info["runs_cheb"], info
        assert np.array_equal(y, y0), (name, mc, np.abs(y - y0).max())
        assert np.array_equal(z, z0), (name, mc, np.abs(z - z0).max())
    # the unstaged operator itself matches the oracle (FP32 tolerance)
    Y = fem.masked_apply(mats, wl["omegas"], wl["rho"], wl["mu"], wl["dir_nodes"], X)
    for k in range(m):
        assert rel_l2(y0[:, k], Y[:, k]) < 1e-5


@pytest.mark.parametrize("stage", [8, 16])
def test_staged_solve_matches_oracle(stage):
    wl = _cases()["pipe"]
    mats = fem.assemble(wl["mesh"])
    X = fem.solve_modes(mats, wl)
    s, mid, rep, u, p = solve(wl, stage=stage, tol=1e-12, max_cycles=2000)
    with s:
        info = scvs.scvs_staged_info(s.ctx, mid)
        Xg = stack_modal(u, p)
    assert info["st_spmm"] == stage and info["st_cheb"] == stage and info["runs_spmm"] and info["runs_cheb"]
    for k, r in enumerate(rep):
        assert r["status"] == scvs.SCVS_CONVERGED, (k, r)
        assert rel_l2(Xg[k], X[k]) < 1e-8, (k, rel_l2(Xg[k], X[k]))


def test_autotuner_times_the_staged_variants():
    wl = _cases()["pipe"]
    s, mid = open_workload(wl, stage=0)
    with s:
        info = scvs.scvs_staged_info(s.ctx, mid)
    assert info["valid"]
    assert all(t > 0 for t in info["spmm_us"][:3]) and all(t > 0 for t in info["cheb_us"][:3])
    assert info["st_spmm"] in (0, 4, 8, 16, 32) and info["st_cheb"] in (0, 4, 8, 16, 32)
