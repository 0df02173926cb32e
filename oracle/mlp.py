"""FP64 CPU oracle of the learned initial guess (test infrastructure only).

The solver's learned guess maps mode features to coefficients of a POD
basis of previously computed solutions.  This module is the plain definition
the GPU kernels are checked against:
  * a multilayer perceptron y = W_3 g(W_2 g(W_1 g(W_0 x + b_0) + b_1) + b_2) + b_3
    with the exact GELU g(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2,
  * its mean-squared-error loss L = sum (y - t)^2 / (B * n_out) over a batch,
  * the gradients of L by reverse-mode differentiation (chain rule written
    out layer by layer),
  * an Adam step (Kingma & Ba 2015: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
    w -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps)),
  * proper orthogonal decomposition by the method of snapshots: eigenvectors
    of the snapshot Gram matrix X^H X, basis Phi = X V Lambda^{-1/2}.
Weights are stored as W_l [in][out] (row = input neuron).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    """d/dz [z Phi(z)] = Phi(z) + z phi(z)."""
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(params, x):
    """params: list of (W [in][out], b [out]); returns output and the
    pre-activations / activations of every layer."""
    acts = [x]
    pres = []
    a = x
    for i, (W, b) in enumerate(params):
        z = a @ W + b
        pres.append(z)
        a = gelu(z) if i < len(params) - 1 else z
        acts.append(a)
    return a, pres, acts


def mse(y, t):
    return float(((y - t) ** 2).sum() / y.size)


def backward(params, x, t):
    """Gradients of mse(forward(x), t) with respect to every W, b."""
    y, pres, acts = forward(params, x)
    delta = 2.0 * (y - t) / y.size
    grads = [None] * len(params)
    for i in range(len(params) - 1, -1, -1):
        W, b = params[i]
        grads[i] = (acts[i].T @ delta, delta.sum(axis=0))
        if i > 0:
            delta = (delta @ W.T) * gelu_grad(pres[i - 1])
    return grads


def adam_step(w, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


def bf16_round(a):
    """Round float64 values to the nearest bfloat16 (round half to even on the
    top 16 bits of the float32 representation)."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def pod(X, n_modes):
    """POD basis of the columns of X (complex, [n][n_snap]) by the method of
    snapshots: X^H X = V Lambda V^H, Phi = X V_r Lambda_r^{-1/2} (orthonormal
    columns, ordered by decreasing energy).  Returns Phi and the eigenvalues."""
    G = X.conj().T @ X
    lam, V = np.linalg.eigh(G)
    order = np.argsort(lam)[::-1]
    lam = lam[order]
    V = V[:, order]
    r = n_modes
    Phi = X @ V[:, :r] / np.sqrt(lam[:r])[None, :]
    return Phi, lam
