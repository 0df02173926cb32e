"""Pins of the MLP / POD oracle of the learned initial guess (no GPU)."""
import math

import numpy as np
import pytest

from oracle import mlp


def _params(rng, sizes, scale=0.3):
    return [(scale * rng.standard_normal((a, b)), 0.1 * rng.standard_normal(b)) for a, b in zip(sizes[:-1], sizes[1:])]


def test_gelu_matches_definition_and_derivative():
    z = np.linspace(-4, 4, 41)
    # z * Phi(z) with Phi from its series-free definition via math.erf
    ref = np.array([v * 0.5 * (1 + math.erf(v / math.sqrt(2))) for v in z])
    assert np.allclose(mlp.gelu(z), ref, atol=1e-15)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.allclose(mlp.gelu_grad(z), fd, atol=1e-8)
    # limits: g(z) -> z for large z, -> 0 for very negative z
    assert abs(mlp.gelu(np.array([10.0]))[0] - 10.0) < 1e-12
    assert abs(mlp.gelu(np.array([-10.0]))[0]) < 1e-12


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    sizes = [5, 7, 6, 6, 4]
    params = _params(rng, sizes)
    x = rng.standard_normal((9, 5))
    t = rng.standard_normal((9, 4))
    grads = mlp.backward(params, x, t)
    h = 1e-6
    for li, (W, b) in enumerate(params):
        for arr, g in ((W, grads[li][0]), (b, grads[li][1])):
            it = np.nditer(arr, flags=["multi_index"])
            for _ in it:
                idx = it.multi_index
                old = arr[idx]
                arr[idx] = old + h
                lp = mlp.mse(mlp.forward(params, x)[0], t)
                arr[idx] = old - h
                lm = mlp.mse(mlp.forward(params, x)[0], t)
                arr[idx] = old
                fd = (lp - lm) / (2 * h)
                assert abs(fd - g[idx]) <= 1e-6 * max(1.0, abs(fd)), (li, idx, fd, g[idx])


def test_adam_minimises_a_quadratic():
    w = np.array([3.0, -2.0])
    m = np.zeros(2)
    v = np.zeros(2)
    # first step moves every coordinate by lr against the sign of the gradient
    w1, m1, v1 = mlp.adam_step(w.copy(), 2 * w, m, v, 1, 0.1)
    assert np.allclose(w1, w - 0.1 * np.sign(w), atol=1e-6)
    for t in range(1, 3000):
        w, m, v = mlp.adam_step(w, 2 * w, m, v, t, 0.01)
    assert np.abs(w).max() < 1e-2


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    a = np.concatenate([rng.standard_normal(1000) * 10.0 ** rng.integers(-5, 5, 1000), [0.0, -0.0, 1.0, 2 ** -20]])
    ref = torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16_round(a), ref)


def test_pod_orthonormal_and_exact_on_low_rank_data():
    rng = np.random.default_rng(3)
    n, r = 200, 5
    B = rng.standard_normal((n, r)) + 1j * rng.standard_normal((n, r))
    C = rng.standard_normal((r, 40)) + 1j * rng.standard_normal((r, 40))
    X = B @ C
    Phi, lam = mlp.pod(X, r)
    assert np.allclose(Phi.conj().T @ Phi, np.eye(r), atol=1e-10)
    # the r-dimensional basis reproduces every snapshot
    rec = Phi @ (Phi.conj().T @ X)
    assert np.abs(rec - X).max() < 1e-9 * np.abs(X).max()
    assert np.all(lam[:r] > 0) and np.all(np.abs(lam[r:]) < 1e-8 * lam[0])
    # eigenvalues are the squared singular values of X
    sv = np.linalg.svd(X, compute_uv=False)
    assert np.allclose(lam[:r], sv[:r] ** 2, rtol=1e-10)


def _spd(rng, n):
    """A sparse-ish real SPD weight like a mass matrix (diagonally dominant band)."""
    import scipy.sparse as spm
    off = 0.2 * rng.random(n - 1)
    d = 1.0 + rng.random(n) + np.r_[off, 0] + np.r_[0, off]
    return spm.diags([off, d, off], [-1, 0, 1], format="csr")


def _snapshots(rng, n=120, r=6, S=30, decay=0.5):
    B = rng.standard_normal((n, r)) + 1j * rng.standard_normal((n, r))
    C = (rng.standard_normal((r, S)) + 1j * rng.standard_normal((r, S))) * decay ** np.arange(r)[:, None]
    return B @ C


def test_weighted_pod_is_orthonormal_in_the_weight_and_matches_the_svd():
    """Phi^H W Phi = I; with W = L L^T the weighted eigenvalues are the squared
    singular values of L^T X (a library routine on a transformed problem)."""
    rng = np.random.default_rng(4)
    n = 120
    W = _spd(rng, n)
    X = _snapshots(rng, n=n) + 0.05 * (rng.standard_normal((n, 30)) + 1j * rng.standard_normal((n, 30)))
    Phi, lam = mlp.pod(X, 8, W)
    assert Phi.shape[1] == 8
    assert np.allclose(Phi.conj().T @ (W @ Phi), np.eye(8), atol=1e-10)
    # Euclidean orthonormality does not hold for a non-trivial weight
    assert np.abs(Phi.conj().T @ Phi - np.eye(8)).max() > 1e-2
    Lt = np.linalg.cholesky(W.toarray()).T
    sv = np.linalg.svd(Lt @ X, compute_uv=False)
    assert np.allclose(lam[:8], sv[:8] ** 2, rtol=1e-9)


def test_weighted_pod_tail_energy_and_phase_convention():
    """The W-norm error of projecting every snapshot onto r vectors is the sum
    of the discarded eigenvalues; for every basis vector, the snapshot with the
    largest coefficient has a real positive coefficient."""
    rng = np.random.default_rng(5)
    n, S = 90, 24
    W = _spd(rng, n)
    X = rng.standard_normal((n, S)) + 1j * rng.standard_normal((n, S))
    for r in (3, 7, 12):
        Phi, lam = mlp.pod(X, r, W)
        A = mlp.pod_coefficients(Phi, X, W)          # [S][r]
        E = X - Phi @ A.T
        err = sum(np.real(np.vdot(E[:, s], W @ E[:, s])) for s in range(S))
        assert abs(err - lam[r:].sum()) < 1e-9 * lam.sum()
        for j in range(r):
            s = int(np.argmax(np.abs(A[:, j])))
            assert A[s, j].real > 0 and abs(A[s, j].imag) < 1e-10 * abs(A[s, j])
    # the rank stops at the numerical rank of low-rank data
    Phi, lam = mlp.pod(_snapshots(rng, n=n, r=4, S=S), 10, W)
    assert Phi.shape[1] == 4


def test_standardise_matches_population_statistics():
    rng = np.random.default_rng(6)
    A = rng.standard_normal((40, 5)) * [1, 2, 3, 0, 5] + [0, 1, 2, 3, 4]
    mu, sd = mlp.standardise(A)
    assert np.allclose(mu, A.mean(axis=0))
    assert np.allclose(sd[[0, 1, 2, 4]], A.std(axis=0, ddof=0)[[0, 1, 2, 4]])
    assert sd[3] == 1.0  # a constant column is left unscaled


def test_learned_guess_reproduces_a_snapshot_from_its_own_coefficients():
    """An MLP whose last layer is zero and whose last bias is the standardised
    target of snapshot s returns that snapshot's projection, which is the
    snapshot itself for data of rank r: pins the (Re, Im) interleaving, the
    block order, the de-standardisation and the expansion."""
    rng = np.random.default_rng(7)
    nu, npr, S, r = 60, 20, 16, 4
    W = _spd(rng, nu)
    Wp = _spd(rng, npr)
    Xu = _snapshots(rng, n=nu, r=r, S=S)
    Xp = _snapshots(rng, n=npr, r=r, S=S)
    Pu, _ = mlp.pod(Xu, r, W)
    Pp, _ = mlp.pod(Xp, r, Wp)
    T = mlp.coefficient_targets(mlp.pod_coefficients(Pu, Xu, W), mlp.pod_coefficients(Pp, Xp, Wp))
    F = rng.standard_normal((S, 5))
    fst, tst = mlp.standardise(F), mlp.standardise(T)
    sizes = [5, 8, 8, 8, 4 * r]
    params = _params(rng, sizes)
    s = 5
    params[-1] = (np.zeros_like(params[-1][0]), (T[s] - tst[0]) / tst[1])
    x = mlp.learned_guess(params, F[[s, s + 1]], fst, tst, Pu, Pp)
    assert np.abs(x[0, :nu] - Xu[:, s]).max() < 1e-10 * np.abs(Xu).max()
    assert np.abs(x[0, nu:] - Xp[:, s]).max() < 1e-10 * np.abs(Xp).max()
    assert np.allclose(x[1], x[0])  # the output no longer depends on the features
