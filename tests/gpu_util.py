"""Helpers shared by the GPU tests: run a workload through the C ABI."""
import numpy as np

from paper_2009_06725_gb300 import scvs


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def open_workload(wl, **opts):
    s = scvs.Solver(**opts)
    mid = scvs.scvs_set_mesh(s.ctx, wl["mesh"])
    scvs.scvs_set_physics(s.ctx, mid, wl["rho"], wl["mu"])
    scvs.scvs_set_modes(s.ctx, mid, wl["omegas"], wl["g"])
    return s, mid


def solve(wl, **opts):
    s, mid = open_workload(wl, **opts)
    m = len(wl["omegas"])
    rep = scvs.scvs_solve(s.ctx, mid, m)
    mesh = wl["mesh"]
    u, p = scvs.scvs_get_modal(s.ctx, mid, m, mesh["xyz"].shape[0], mesh["dim"], mesh["n_vertices"])
    return s, mid, rep, u, p


def stack_modal(u, p):
    """[m][N][d], [m][P] -> [m][n_dof] in the oracle's dof order."""
    m = u.shape[0]
    return np.concatenate([u.reshape(m, -1), p], axis=1)


def padded_block(X, ld):
    """[n][m] -> [n][ld] with zero padding columns."""
    n, m = X.shape
    out = np.zeros((n, ld), dtype=X.dtype)
    out[:, :m] = X
    return out


def apply_gpu(s, mid, X, precision, matfree=False):
    torch = torch_cuda()
    ld = scvs.scvs_mode_stride(s.ctx, mid)
    Xp = padded_block(X, ld)
    dt = torch.complex128 if precision == scvs.SCVS_PREC_FP64 else torch.complex64
    x = torch.from_numpy(Xp).to(dt).cuda()
    y = torch.zeros_like(x)
    torch.cuda.synchronize()
    f = scvs.scvs_apply_matfree if matfree else scvs.scvs_apply
    f(s.ctx, mid, precision, x.data_ptr(), y.data_ptr())
    torch.cuda.synchronize()
    return y.cpu().numpy().astype(np.complex128)[:, : X.shape[1]]


def rel_err(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
