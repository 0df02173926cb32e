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
