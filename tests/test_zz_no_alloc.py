"""The allocation-free reconstruction entry point agrees with the allocating one.

scvs_reconstruct_dev_static serves callers that must not allocate device
memory during a call: code that runs while a framework's caching allocator
holds nearly all of the GPU's memory (a cudaMalloc could fail or fragment
it) and latency-critical pipelines that cannot take the device-wide
synchronisation of cudaMalloc/cudaFree.  Its twiddle scratch is a fixed
file-scope device table instead of a per-call buffer.  This file is named so
that pytest collects it last.
"""
import numpy as np
import pytest

from paper_2009_06725_gb300 import scvs
from synthetic import workloads

from .gpu_util import rel_err, solve, torch_cuda

pytestmark = pytest.mark.gpu


def test_static_reconstruction_matches_allocating_entry_point():
    torch = torch_cuda()
    wl = workloads.channel_workload(32, 8, n_modes=8)
    s, mid, rep, u, p = solve(wl, precision=scvs.SCVS_PREC_FP64, tol=1e-12)
    N, P = u.shape[1], p.shape[1]
    with s:
        # two calls in a row, with different sample counts and periods
        for n_t, period in ((24, 1.0), (40, 2.0)):
            ref_u = torch.zeros((n_t, N, 2), dtype=torch.float64, device="cuda")
            ref_p = torch.zeros((n_t, P), dtype=torch.float64, device="cuda")
            out_u = torch.full_like(ref_u, float("nan"))
            out_p = torch.full_like(ref_p, float("nan"))
            torch.cuda.synchronize()
            scvs.scvs_reconstruct_dev(s.ctx, mid, n_t, period, ref_u.data_ptr(), ref_p.data_ptr())
            scvs.scvs_reconstruct_dev_static(s.ctx, mid, n_t, period, out_u.data_ptr(), out_p.data_ptr())
            torch.cuda.synchronize()
            a, b = out_u.cpu().numpy(), ref_u.cpu().numpy()
            assert np.all(np.isfinite(a))
            assert rel_err(a, b) < 1e-12
            assert rel_err(out_p.cpu().numpy(), ref_p.cpu().numpy()) < 1e-12
        # sizes beyond the static table are refused with a clear error
        too_many = scvs.SCVS_RECON_STATIC_MAX // 8 + 1
        big_u = torch.empty((1,), dtype=torch.float64, device="cuda")
        with pytest.raises(scvs.ScvsError) as e:
            scvs.scvs_reconstruct_dev_static(s.ctx, mid, too_many, 1.0, big_u.data_ptr(), big_u.data_ptr())
        assert e.value.code == scvs.SCVS_ERR_ARG
        assert "SCVS_RECON_STATIC_MAX" in str(e.value)


def test_static_reconstruction_allocates_nothing():
    """A warm call leaves the context pool's high-water mark, its reservation
    and the device's free memory unchanged and launches exactly its two
    kernels; the allocating entry point, timed the same way, raises the
    high-water mark (so the probe can see an allocation)."""
    torch = torch_cuda()
    wl = workloads.channel_workload(16, 4, n_modes=8)
    s, mid, rep, u, p = solve(wl, precision=scvs.SCVS_PREC_FP64, tol=1e-12)
    N, P = u.shape[1], p.shape[1]
    n_t = 32
    with s:
        out_u = torch.zeros((n_t, N, 2), dtype=torch.float64, device="cuda")
        out_p = torch.zeros((n_t, P), dtype=torch.float64, device="cuda")
        scvs.scvs_reconstruct_dev_static(s.ctx, mid, n_t, 1.0, out_u.data_ptr(), out_p.data_ptr())  # set-up call
        torch.cuda.synchronize()
        used0, _, res0 = scvs.scvs_pool_usage(s.ctx, reset_high=True)
        free0 = torch.cuda.mem_get_info()[0]
        n0 = scvs.scvs_launch_count(s.ctx)
        scvs.scvs_reconstruct_dev_static(s.ctx, mid, n_t, 1.0, out_u.data_ptr(), out_p.data_ptr())
        torch.cuda.synchronize()
        used1, high1, res1 = scvs.scvs_pool_usage(s.ctx, reset_high=True)
        free1 = torch.cuda.mem_get_info()[0]
        assert scvs.scvs_launch_count(s.ctx) == n0 + 2
        assert (used1, high1, res1) == (used0, used0, res0)
        assert free1 == free0
        # the same probe around the allocating entry point sees its scratch
        scvs.scvs_reconstruct_dev(s.ctx, mid, n_t, 1.0, out_u.data_ptr(), out_p.data_ptr())
        used2, high2, _ = scvs.scvs_pool_usage(s.ctx)
        assert used2 == used0 and high2 > used0
