"""Learned initial guess on the GPU: MLP kernels against the FP64 oracle
(same BF16-rounded weights; the GPU accumulates in FP32), Adam against the
oracle step, and the trained guess against zero-start GMRES."""
import numpy as np
import pytest

from oracle import mlp as omlp
from paper_2009_06725_gb300 import scvs
from synthetic import workloads

from .gpu_util import torch_cuda

pytestmark = pytest.mark.gpu

SIZES = [5, 256, 256, 256, 40]


def _flat(params):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in params]).astype(np.float32)


def _unflat(v, sizes):
    out, o = [], 0
    for a, b in zip(sizes[:-1], sizes[1:]):
        W = v[o:o + a * b].reshape(a, b)
        o += a * b
        out.append((W, v[o:o + b]))
        o += b
    return out


def _setup(seed=0, B=48):
    rng = np.random.default_rng(seed)
    params = [(rng.standard_normal((a, b)) * np.sqrt(2.0 / a), 0.1 * rng.standard_normal(b))
              for a, b in zip(SIZES[:-1], SIZES[1:])]
    flat = _flat(params)
    rounded = [(omlp.bf16_round(W), omlp.bf16_round(b)) for W, b in _unflat(flat.astype(np.float64), SIZES)]
    x = rng.standard_normal((B, SIZES[0])).astype(np.float32)
    t = rng.standard_normal((B, SIZES[-1])).astype(np.float32)
    return flat, rounded, x, t


def test_mlp_forward_and_gradient_match_oracle():
    torch = torch_cuda()
    flat, rounded, x, t = _setup()
    B = x.shape[0]
    with scvs.Solver() as s:
        scvs.scvs_mlp_init(s.ctx, SIZES[0], SIZES[1], SIZES[-1], flat)
        xd = torch.from_numpy(x).cuda()
        td = torch.from_numpy(t).cuda()
        yd = torch.empty((B, SIZES[-1]), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        scvs.scvs_mlp_forward_dev(s.ctx, xd.data_ptr(), B, yd.data_ptr())
        torch.cuda.synchronize()
        g, loss = scvs.scvs_mlp_gradient_dev(s.ctx, xd.data_ptr(), td.data_ptr(), B)
        y = yd.cpu().numpy()
    yr, _, _ = omlp.forward(rounded, x.astype(np.float64))
    assert np.abs(y - yr).max() < 1e-4 * np.abs(yr).max()
    assert abs(loss - omlp.mse(yr, t)) < 1e-4 * omlp.mse(yr, t)
    gr = omlp.backward(rounded, x.astype(np.float64), t.astype(np.float64))
    gg = _unflat(g.astype(np.float64), SIZES)
    for (gw, gb), (rw, rb) in zip(gg, gr):
        assert np.abs(gw - rw).max() < 1e-3 * np.abs(rw).max()
        assert np.abs(gb - rb).max() < 1e-3 * np.abs(rb).max()


def test_adam_step_matches_oracle():
    torch = torch_cuda()
    flat, rounded, x, t = _setup(seed=1, B=32)
    with scvs.Solver() as s:
        scvs.scvs_mlp_init(s.ctx, SIZES[0], SIZES[1], SIZES[-1], flat)
        xd = torch.from_numpy(x).cuda()
        td = torch.from_numpy(t).cuda()
        torch.cuda.synchronize()
        g, _ = scvs.scvs_mlp_gradient_dev(s.ctx, xd.data_ptr(), td.data_ptr(), x.shape[0])
        scvs.scvs_mlp_adam_step(s.ctx, 1e-3)
        after = scvs.scvs_mlp_get_params(s.ctx)
    w = flat.astype(np.float64)
    ref, _, _ = omlp.adam_step(w, g.astype(np.float64), np.zeros_like(w), np.zeros_like(w), 1, 1e-3)
    assert np.abs(after - ref).max() < 1e-6


def _family(n_geo, seed, n_modes=16):
    rng = np.random.default_rng(seed)
    out = []
    for gi in range(n_geo):
        R = rng.uniform(0.7, 1.3)
        st = rng.uniform(0.0, 0.4)
        wl = workloads.pipe_workload(n_c=3, n_r=2, n_x=6, n_modes=n_modes, length=3.0, radius=R, stenosis=st,
                                     seed=0)
        # per-geometry phases of the inlet coefficients
        c = workloads.phases(n_modes, seed=1000 + 97 * seed + gi)
        g = wl["g"] / wl["coeffs"][:, None, None] * c[:, None, None]
        wl = dict(wl, coeffs=c, g=g)
        feats = np.stack([wl["omegas"], c.real, c.imag, np.full(n_modes, R), np.full(n_modes, st)], axis=1)
        out.append((wl, feats))
    return out


def test_learned_guess_reduces_iterations():
    train = _family(12, seed=0)
    test = _family(3, seed=1)
    conn0 = train[0][0]["mesh"]["conn"]
    for wl, _ in train + test:
        assert np.array_equal(wl["mesh"]["conn"], conn0)  # morphs share the node set
    with scvs.Solver() as s:
        for wl, f in train:
            scvs.scvs_clear_meshes(s.ctx)
            mid = scvs.scvs_set_mesh(s.ctx, wl["mesh"])
            scvs.scvs_set_physics(s.ctx, mid, wl["rho"], wl["mu"])
            scvs.scvs_set_modes(s.ctx, mid, wl["omegas"], wl["g"])
            rep = scvs.scvs_solve(s.ctx, mid, len(f))
            assert all(r["status"] == scvs.SCVS_CONVERGED for r in rep)
            scvs.scvs_guess_add_snapshots(s.ctx, mid, f)
        info = scvs.scvs_guess_info(s.ctx)
        assert info["n_snapshots"] == 12 * 16
        loss = scvs.scvs_train_guess(s.ctx, scvs.scvs_default_train_opts(n_pod=16, steps=1500, batch=64))
        assert np.isfinite(loss)
        it0, it1, used, res0 = [], [], [], []
        for wl, f in test:
            res = {}
            for guess in (scvs.SCVS_GUESS_ZERO, scvs.SCVS_GUESS_MLP):
                s.set_opts(guess=guess)
                scvs.scvs_clear_meshes(s.ctx)
                mid = scvs.scvs_set_mesh(s.ctx, wl["mesh"])
                scvs.scvs_set_physics(s.ctx, mid, wl["rho"], wl["mu"])
                scvs.scvs_set_modes(s.ctx, mid, wl["omegas"], wl["g"])
                scvs.scvs_guess_set_features(s.ctx, mid, f)
                rep = scvs.scvs_solve(s.ctx, mid, len(f))
                assert all(r["status"] == scvs.SCVS_CONVERGED for r in rep)
                u, p = scvs.scvs_get_modal(s.ctx, mid, len(f), wl["mesh"]["xyz"].shape[0], 3, wl["mesh"]["n_vertices"])
                res[guess] = (rep, np.concatenate([u.reshape(len(f), -1), p], axis=1))
            it0 += [r["iterations"] for r in res[scvs.SCVS_GUESS_ZERO][0]]
            it1 += [r["iterations"] for r in res[scvs.SCVS_GUESS_MLP][0]]
            used += [r["guess_used"] for r in res[scvs.SCVS_GUESS_MLP][0]]
            res0 += [r["res0"] for r in res[scvs.SCVS_GUESS_MLP][0] if r["guess_used"]]
            assert all(abs(r["res0"] - 1.0) < 1e-12 for r in res[scvs.SCVS_GUESS_ZERO][0])
            X0, X1 = res[scvs.SCVS_GUESS_ZERO][1], res[scvs.SCVS_GUESS_MLP][1]
            for k in range(len(f)):
                assert np.linalg.norm(X1[k] - X0[k]) <= 1e-6 * np.linalg.norm(X0[k])
    # the guess is kept on most held-out modes, starts well inside the zero
    # start's residual and saves Arnoldi steps
    assert sum(used) >= len(used) // 2, used
    assert np.median(res0) < 0.5, res0
    assert np.mean(it1) < np.mean(it0), (np.mean(it0), np.mean(it1))
