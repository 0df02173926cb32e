"""The learned guess's POD and expansion on the GPU against the oracle.

Both sides take the snapshots of the same seeded family of pipe morphs (the
GPU from its own FP64 solves, the oracle from its sparse LU), form the POD of
each field block in the block's L2(Omega) inner product (the reference
geometry's mass matrices) with the same phase convention, and expand the
same seeded MLP weights into x0 = c_k [Phi_u a_u; Phi_p a_p] with g on the
Dirichlet rows.  Compared element by element: the bases, the snapshot
coefficients, x0, its residual and the solver's keep / fall-back decision."""
import numpy as np
import pytest

from oracle import fem
from oracle import mlp as omlp
from paper_2009_06725_gb300 import scvs
from synthetic import workloads

pytestmark = pytest.mark.gpu

N_MODES, N_GEO, N_POD, HIDDEN = 8, 4, 6, 32


def _family():
    rng = np.random.default_rng(0)
    out = []
    for gi in range(N_GEO):
        R = rng.uniform(0.7, 1.3)
        st = rng.uniform(0.0, 0.4)
        wl = workloads.pipe_workload(n_c=3, n_r=2, n_x=6, n_modes=N_MODES, length=3.0, radius=R, stenosis=st, seed=0)
        c = workloads.phases(N_MODES, seed=1000 + gi)
        g = wl["g"] / wl["coeffs"][:, None, None] * c[:, None, None]
        wl = dict(wl, coeffs=c, g=g)
        feats = np.stack([wl["omegas"], c.real, c.imag, np.full(N_MODES, R), np.full(N_MODES, st)], axis=1)
        out.append((wl, feats))
    return out


@pytest.fixture(scope="module")
def family():
    fam = _family()
    mats0 = fem.assemble(fam[0][0]["mesh"])
    Wu, Wp = fem.block_weights(mats0, fam[0][0]["mesh"])
    snaps, feats = [], []
    for wl, f in fam:
        X = fem.solve_modes(fem.assemble(wl["mesh"]), wl)
        snaps += [X[k] / wl["coeffs"][k] for k in range(N_MODES)]
        feats.append(f)
    X = np.array(snaps).T                       # [n_dof][S]
    nu = 3 * mats0["N"]
    Pu, lam_u = omlp.pod(X[:nu], N_POD, Wu)
    Pp, lam_p = omlp.pod(X[nu:], N_POD, Wp)
    au, ap = omlp.pod_coefficients(Pu, X[:nu], Wu), omlp.pod_coefficients(Pp, X[nu:], Wp)
    F = np.concatenate(feats)
    T = omlp.coefficient_targets(au, ap)
    return dict(fam=fam, mats0=mats0, Wu=Wu, Wp=Wp, nu=nu, Pu=Pu, Pp=Pp, au=au, ap=ap,
                fst=omlp.standardise(F), tst=omlp.standardise(T), T=T)


def _trained_solver(fam):
    s = scvs.Solver(precision=scvs.SCVS_PREC_FP64, tol=1e-12)
    for wl, f in fam:
        scvs.scvs_clear_meshes(s.ctx)
        mid = scvs.scvs_set_mesh(s.ctx, wl["mesh"])
        scvs.scvs_set_physics(s.ctx, mid, wl["rho"], wl["mu"])
        scvs.scvs_set_modes(s.ctx, mid, wl["omegas"], wl["g"])
        rep = scvs.scvs_solve(s.ctx, mid, N_MODES)
        assert all(r["status"] == scvs.SCVS_CONVERGED for r in rep)
        scvs.scvs_guess_add_snapshots(s.ctx, mid, f)
    # POD and standardisation only: no Adam step, the weights are set below
    scvs.scvs_train_guess(s.ctx, scvs.scvs_default_train_opts(n_pod=N_POD, hidden=HIDDEN, steps=0,
                                                             max_pod_snapshots=N_GEO * N_MODES))
    return s


def _col_err(A, B):
    return max(np.abs(A[:, j] - B[:, j]).max() / np.abs(B[:, j]).max() for j in range(B.shape[1]))


def test_pod_basis_and_coefficients_match_oracle(family):
    with _trained_solver(family["fam"]) as s:
        info = scvs.scvs_guess_info(s.ctx)
        assert info["n_pod"] == N_POD and info["n_snapshots"] == N_GEO * N_MODES
        nu = family["nu"]
        Gu = scvs.scvs_guess_basis(s.ctx, 0, nu)
        Gp = scvs.scvs_guess_basis(s.ctx, 1, family["Pp"].shape[0])
        cu, cp = scvs.scvs_guess_coefficients(s.ctx, 0), scvs.scvs_guess_coefficients(s.ctx, 1)
    # the GPU basis is orthonormal in the oracle's mass inner products
    assert np.abs(Gu.conj().T @ (family["Wu"] @ Gu) - np.eye(N_POD)).max() < 1e-4
    assert np.abs(Gp.conj().T @ (family["Wp"] @ Gp) - np.eye(N_POD)).max() < 1e-4
    # element by element, phases included (both sides fix them the same way)
    assert _col_err(Gu, family["Pu"]) < 2e-3
    assert _col_err(Gp, family["Pp"]) < 2e-3
    # coefficients against the size of the snapshot's whole coefficient vector (the error of the
    # reconstruction Phi a): a weak vector's own coefficients are ill-conditioned, because FP32
    # snapshots tilt it towards the dominant directions by ~eps_32 sigma_1 / sigma_j
    for A, B in ((cu, family["au"]), (cp, family["ap"])):
        assert (np.abs(A - B).max(axis=1) / np.abs(B).max(axis=1)).max() < 1e-4
    # the leading vectors, whose eigenvalues stand well apart, agree closely
    assert _col_err(Gu[:, :3], family["Pu"][:, :3]) < 1e-4
    assert _col_err(cu[:, :3], family["au"][:, :3]) < 1e-4


def _flat(params):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in params]).astype(np.float32)


def _rounded(flat, sizes):
    out, o = [], 0
    v = flat.astype(np.float64)
    for a, b in zip(sizes[:-1], sizes[1:]):
        W = v[o:o + a * b].reshape(a, b)
        o += a * b
        out.append((omlp.bf16_round(W), omlp.bf16_round(v[o:o + b])))
        o += b
    return out


def _oracle_x0(family, params, wl, feats):
    """x0 of every mode by the definition: c_k times the expansion, g on the
    Dirichlet rows."""
    X0 = omlp.learned_guess(params, feats, family["fst"], family["tst"], family["Pu"], family["Pp"])
    X0 = X0 * wl["coeffs"][:, None]
    dd = fem.dirichlet_dofs(wl["dir_nodes"], 3)
    for k in range(N_MODES):
        X0[k, dd] = wl["g"][k].reshape(-1)
    return X0


def _probe(s, wl, feats):
    scvs.scvs_clear_meshes(s.ctx)
    mid = scvs.scvs_set_mesh(s.ctx, wl["mesh"])
    scvs.scvs_set_physics(s.ctx, mid, wl["rho"], wl["mu"])
    scvs.scvs_set_modes(s.ctx, mid, wl["omegas"], wl["g"])
    scvs.scvs_guess_set_features(s.ctx, mid, feats)
    res0, kept = scvs.scvs_guess_initial(s.ctx, mid, N_MODES)
    mesh = wl["mesh"]
    u, p = scvs.scvs_get_modal(s.ctx, mid, N_MODES, mesh["xyz"].shape[0], 3, mesh["n_vertices"])
    return mid, res0, kept, np.concatenate([u.reshape(N_MODES, -1), p], axis=1)


def test_expanded_guess_matches_oracle(family):
    sizes = [5, HIDDEN, HIDDEN, HIDDEN, 4 * N_POD]
    rng = np.random.default_rng(11)
    params = [(rng.standard_normal((a, b)) * np.sqrt(1.0 / a), 0.1 * rng.standard_normal(b))
              for a, b in zip(sizes[:-1], sizes[1:])]
    flat = _flat(params)
    wl, feats = family["fam"][1]
    with _trained_solver(family["fam"]) as s:
        assert scvs.scvs_mlp_num_params(s.ctx) == flat.size
        scvs.scvs_mlp_set_params(s.ctx, flat)
        _, res0, kept, X0g = _probe(s, wl, feats)
    X0 = _oracle_x0(family, _rounded(flat, sizes), wl, feats)
    dd = fem.dirichlet_dofs(wl["dir_nodes"], 3)
    for k in range(N_MODES):
        assert np.linalg.norm(X0g[k] - X0[k]) < 2e-3 * np.linalg.norm(X0[k]), k
        assert np.array_equal(X0g[k, dd], X0[k, dd])        # Dirichlet rows are g, exactly
    r_or = fem.relative_residual(fem.assemble(wl["mesh"]), wl, X0)
    assert np.all(np.abs(res0 - r_or) < 2e-3 * np.maximum(r_or, 1.0)), (res0, r_or)
    clear = np.abs(r_or - 1.0) > 1e-2                      # decisions far from the threshold
    assert np.array_equal(kept[clear], (r_or < 1.0)[clear])


def test_keep_and_fallback_decisions(family):
    """A network whose output is the standardised target of snapshot s returns
    that snapshot's POD projection: kept for the mode it came from, with the
    residual the solve reports; a huge output is dropped for every mode and
    the solve starts from zero."""
    wl, feats = family["fam"][0]
    k = 3                                                  # snapshot s = k of the reference geometry
    sizes = [5, HIDDEN, HIDDEN, HIDDEN, 4 * N_POD]
    rng = np.random.default_rng(12)
    params = [(rng.standard_normal((a, b)) * np.sqrt(1.0 / a), 0.1 * rng.standard_normal(b))
              for a, b in zip(sizes[:-1], sizes[1:])]
    params[-1] = (np.zeros_like(params[-1][0]), (family["T"][k] - family["tst"][0]) / family["tst"][1])
    with _trained_solver(family["fam"]) as s:
        scvs.scvs_mlp_set_params(s.ctx, _flat(params))
        mid, res0, kept, X0g = _probe(s, wl, feats)
        X0 = _oracle_x0(family, _rounded(_flat(params), sizes), wl, feats)
        assert np.linalg.norm(X0g[k] - X0[k]) < 2e-3 * np.linalg.norm(X0[k])
        assert kept[k] and res0[k] < 0.1, res0
        s.set_opts(guess=scvs.SCVS_GUESS_MLP)
        rep = scvs.scvs_solve(s.ctx, mid, N_MODES)
        assert rep[k]["guess_used"] == 1 and abs(rep[k]["res0"] - res0[k]) < 1e-12 * max(res0[k], 1e-300) + 1e-15
        for j in range(N_MODES):
            assert rep[j]["guess_used"] == int(kept[j])
        # a useless guess: every mode falls back to the zero start
        big = [(W, b) for W, b in params]
        big[-1] = (big[-1][0], big[-1][1] + 1e6)
        scvs.scvs_mlp_set_params(s.ctx, _flat(big))
        mid, res0, kept, _ = _probe(s, wl, feats)
        assert not kept.any() and np.all(res0 > 1.0)
        s.set_opts(guess=scvs.SCVS_GUESS_MLP)
        rep = scvs.scvs_solve(s.ctx, mid, N_MODES)
        assert all(r["guess_used"] == 0 and abs(r["res0"] - 1.0) < 1e-12 for r in rep)
        assert all(r["status"] == scvs.SCVS_CONVERGED for r in rep)
