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
  * proper orthogonal decomposition by the method of snapshots in the
    L2(Omega) inner product of the field block (Gram matrix X^H W X with W
    the block's mass matrix), basis Phi = X V Lambda^{-1/2}, so that
    Phi^H W Phi = I; each eigenvector is scaled by a unit complex number
    that makes its entry of largest magnitude real and positive (this fixes
    the phase of every basis vector), and the coefficients of a snapshot x
    are a = Phi^H W x,
  * the learned initial guess of a mode: standardised features through the
    MLP, de-standardised outputs read as the POD coefficients of x / c_k,
    x0 = c_k [Phi_u a_u; Phi_p a_p], Dirichlet dofs reset to g, and the
    zero-start fallback when the guess's residual is not below ||b||.
Weights are stored as W_l [in][out] (row = input neuron).

The POD, the standardisation and the guess have no counterpart in the
paper: they define the learned part of the solver (features of Eq.
stokes_complex's data: omega_k, the boundary coefficient c_k and the
geometry).
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


def pod(X, n_modes, W=None, rel_floor=1e-10):
    """POD basis of the columns of X (complex, [n][n_snap]) by the method of
    snapshots in the inner product <x, y> = x^H W y (W = identity if None):
    X^H W X = V Lambda V^H with eigenvalues descending, each column of V
    scaled so that its largest-magnitude entry is real positive, and
    Phi = X V_r Lambda_r^{-1/2} with r = min(n_modes, #{lambda_i > rel_floor
    lambda_1}).  Returns Phi [n][r] (W-orthonormal columns) and every
    eigenvalue."""
    WX = X if W is None else W @ X
    G = X.conj().T @ WX
    G = 0.5 * (G + G.conj().T)
    lam, V = np.linalg.eigh(G)
    order = np.argsort(lam)[::-1]
    lam = lam[order]
    V = V[:, order]
    r = 0
    while r < min(n_modes, lam.size) and lam[r] > rel_floor * lam[0]:
        r += 1
    V = V[:, :r].copy()
    for j in range(r):
        i = int(np.argmax(np.abs(V[:, j])))
        V[:, j] *= np.conj(V[i, j]) / abs(V[i, j])
    Phi = X @ V / np.sqrt(lam[:r])[None, :]
    return Phi, lam


def pod_coefficients(Phi, X, W=None):
    """Coefficients of the snapshots X [n][S] in the basis Phi: a = Phi^H W x,
    returned as [S][r]."""
    WX = X if W is None else W @ X
    return (Phi.conj().T @ WX).T


def standardise(A):
    """Column means and population standard deviations of A [S][q] as the
    learned guess uses them (a deviation of zero is replaced by one)."""
    mu = A.mean(axis=0)
    sd = np.sqrt(((A - mu) ** 2).mean(axis=0))
    return mu, np.where(sd > 1e-12, sd, 1.0)


def coefficient_targets(au, ap):
    """Training targets [S][4r] from the block coefficients [S][r]:
    (Re a_u,0, Im a_u,0, Re a_u,1, ...) then the same for the pressure."""
    S, r = au.shape
    T = np.empty((S, 4 * r))
    T[:, 0:2 * r:2] = au.real
    T[:, 1:2 * r:2] = au.imag
    T[:, 2 * r::2] = ap.real
    T[:, 2 * r + 1::2] = ap.imag
    return T


def learned_guess(params, feats, fstats, tstats, Phi_u, Phi_p):
    """x0 / c_k of every mode before the Dirichlet reset: the MLP maps the
    standardised features [m][5] to standardised coefficients, which are
    de-standardised and expanded in the two POD bases.  Returns [m][n_u + n_p]."""
    z = (feats - fstats[0]) / fstats[1]
    y, _, _ = forward(params, z)
    t = y * tstats[1] + tstats[0]
    r = Phi_u.shape[1]
    au = t[:, 0:2 * r:2] + 1j * t[:, 1:2 * r:2]
    ap = t[:, 2 * r::2] + 1j * t[:, 2 * r + 1::2]
    return np.concatenate([au @ Phi_u.T, ap @ Phi_p.T], axis=1)
