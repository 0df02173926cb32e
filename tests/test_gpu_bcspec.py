"""Spectral preprocessing of sampled boundary data on the GPU (Eqs. SCVS_bc,
mode_error) against the FP64 oracle, its output used as the solver's per-mode
Dirichlet data (steps 1-3 of the algorithm of Sec. 3), and the a posteriori
mode energies of a solved mesh."""
import numpy as np
import pytest

from oracle import bcspec, fem
from paper_2009_06725_gb300 import scvs
from synthetic import workloads

from .gpu_util import rel_l2, stack_modal, torch_cuda

pytestmark = pytest.mark.gpu


def _samples(wl, n_t, seed=0):
    """Inlet data of mode 1's Womersley shape times a periodic waveform with an
    infinite but fast-decaying spectrum (exp(cos)) plus a few seeded harmonics;
    walls stay zero.  Returns g_t [n_t][n_dir][3]."""
    rng = np.random.default_rng(seed)
    shape = np.abs(wl["g"][1]) / max(np.abs(wl["g"][1]).max(), 1e-300)  # [n_dir][3], zero on walls
    t = np.arange(n_t) / n_t
    a = np.exp(np.cos(2 * np.pi * t))
    for k in range(1, 4):
        a += rng.uniform(0.1, 0.5) * np.cos(2 * np.pi * k * t + rng.uniform(0, 2 * np.pi))
    return a[:, None, None] * shape[None]


@pytest.mark.parametrize("weighted", [False, True])
def test_spectrum_matches_oracle(weighted):
    torch = torch_cuda()
    wl = workloads.pipe_workload(n_c=3, n_r=2, n_x=6, n_modes=2, length=3.0)
    n_t, m = 64, 12
    g_t = _samples(wl, n_t)
    n_pts = g_t[0].size
    w = np.random.default_rng(5).uniform(0.5, 2.0, n_pts) if weighted else np.ones(n_pts)
    gd = torch.from_numpy(g_t.reshape(n_t, n_pts)).cuda()
    wd = torch.from_numpy(w).cuda() if weighted else None
    cd = torch.zeros((m, n_pts), dtype=torch.complex128, device="cuda")
    with scvs.Solver() as s:
        torch.cuda.synchronize()
        e2 = scvs.scvs_bc_spectrum(s.ctx, gd.data_ptr(), n_t, n_pts, m, cd.data_ptr(),
                                   wd.data_ptr() if weighted else None)
        torch.cuda.synchronize()
    c = cd.cpu().numpy()
    ref_c = bcspec.solver_modes(bcspec.fourier_coefficients(g_t.reshape(n_t, n_pts), m))
    assert np.abs(c - ref_c).max() < 1e-13 * np.abs(ref_c).max()
    ref_e2 = bcspec.truncation_errors([(g_t.reshape(n_t, n_pts), w)], m)
    assert np.allclose(e2, ref_e2, rtol=1e-9, atol=1e-14), (e2, ref_e2)
    N, _ = bcspec.select_modes([(g_t.reshape(n_t, n_pts), w)], 1e-4, m)
    assert N is not None and np.sqrt(e2[N]) < 1e-4 <= np.sqrt(e2[N - 1])


def test_spectrum_feeds_the_solve():
    torch = torch_cuda()
    wl = workloads.pipe_workload(n_c=3, n_r=2, n_x=6, n_modes=2, length=3.0)
    n_t, m = 48, 6
    g_t = _samples(wl, n_t, seed=1)
    n_dir = g_t.shape[1]
    n_pts = n_dir * 3
    gd = torch.from_numpy(g_t.reshape(n_t, n_pts)).cuda()
    cd = torch.zeros((m, n_pts), dtype=torch.complex128, device="cuda")
    omegas = 2 * np.pi * np.arange(m) / wl["period"]
    with scvs.Solver(tol=1e-12, max_cycles=2000) as s:
        mid = scvs.scvs_set_mesh(s.ctx, wl["mesh"])
        scvs.scvs_set_physics(s.ctx, mid, wl["rho"], wl["mu"])
        torch.cuda.synchronize()
        scvs.scvs_bc_spectrum(s.ctx, gd.data_ptr(), n_t, n_pts, m, cd.data_ptr())
        scvs.scvs_set_modes_dev(s.ctx, mid, omegas, cd.data_ptr())
        rep = scvs.scvs_solve(s.ctx, mid, m)
        mesh = wl["mesh"]
        u, p = scvs.scvs_get_modal(s.ctx, mid, m, mesh["xyz"].shape[0], 3, mesh["n_vertices"])
    assert all(r["status"] == scvs.SCVS_CONVERGED for r in rep), rep
    c = bcspec.solver_modes(bcspec.fourier_coefficients(g_t.reshape(n_t, n_pts), m)).reshape(m, n_dir, 3)
    X = fem.solve_modes(fem.assemble(wl["mesh"]), dict(wl, omegas=omegas, g=c))
    Xg = stack_modal(u, p)
    for k in range(m):
        assert rel_l2(Xg[k], X[k]) < 1e-8, k


def test_bad_sizes():
    torch = torch_cuda()
    gd = torch.zeros((8, 3), dtype=torch.float64, device="cuda")
    cd = torch.zeros((8, 3), dtype=torch.complex128, device="cuda")
    with scvs.Solver() as s:
        for n_t, m in ((8, 5), (1, 1), (8, 0)):
            with pytest.raises(scvs.ScvsError) as e:
                scvs.scvs_bc_spectrum(s.ctx, gd.data_ptr(), n_t, 3, m, cd.data_ptr())
            assert e.value.code == scvs.SCVS_ERR_ARG


def test_mode_energies_match_oracle():
    """Energies and a posteriori increments of a solved mesh and of a batch of two
    components, against the oracle's literal time-domain evaluation on the GPU's
    own modal solution."""
    wls = [workloads.pipe_workload(n_c=3, n_r=2, n_x=5, n_modes=6, length=2.5, seed=0),
           workloads.pipe_workload(n_c=2, n_r=1, n_x=4, n_modes=6, length=2.0, radius=0.8, seed=1)]
    U = workloads.union_workload(wls)
    m = len(U["omegas"])
    with scvs.Solver(tol=1e-12, max_cycles=2000) as s:
        mid = scvs.scvs_set_mesh(s.ctx, U["mesh"])
        scvs.scvs_set_components(s.ctx, mid, U["n_comp"], U["node_comp"])
        scvs.scvs_set_physics(s.ctx, mid, U["rho"], U["mu"])
        with pytest.raises(scvs.ScvsError) as e:
            scvs.scvs_mode_energies(s.ctx, mid, 2 * m)
        assert e.value.code == scvs.SCVS_ERR_STATE
        scvs.scvs_set_modes(s.ctx, mid, U["omegas"], U["g"])
        rep = scvs.scvs_solve(s.ctx, mid, 2 * m)
        assert all(r["status"] == scvs.SCVS_CONVERGED for r in rep)
        E, inc = scvs.scvs_mode_energies(s.ctx, mid, 2 * m)
        N = U["mesh"]["xyz"].shape[0]
        u, _ = scvs.scvs_get_modal(s.ctx, mid, m, N, 3, U["mesh"]["n_vertices"])
    for i, (wl, mp) in enumerate(zip(wls, U["maps"])):
        Ms = fem.assemble(wl["mesh"])["Ms"]
        Ui = u[:, mp]
        ref_E = bcspec.mode_energies(Ms, Ui, U["omegas"], U["period"], 32)
        ref_inc = bcspec.a_posteriori_increments(Ms, Ui, U["omegas"], U["period"], 32)
        assert np.allclose(E[i * m:(i + 1) * m], ref_E, rtol=1e-11, atol=0), (i, E, ref_E)
        assert np.allclose(inc[i * m:(i + 1) * m], ref_inc, rtol=1e-10, atol=1e-15), (i, inc, ref_inc)
