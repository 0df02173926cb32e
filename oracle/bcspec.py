"""FP64 CPU oracle of the spectral preprocessing of the boundary data (test
infrastructure: only the tests, ``__graft_entry__.smoke`` and the CPU-baseline
leg of ``bench.py`` use it; it imports nothing from the product).

What it computes (arXiv 2009.06725, Sec. 3, steps 1 and 2 of the algorithm):
  * the Fourier coefficients of a periodic boundary field,
    g~_i = (1/T) int_0^T g(t) e^{-j omega_i t} dt (Eq. SCVS_bc), with omega_i =
    2 pi i / T, from n_t uniform samples t_s = s T / n_t by the rectangle rule
    (exact for trigonometric polynomials of degree below n_t / 2);
  * the per-mode Dirichlet data of the solver, c_0 = g~_0 and c_i = 2 g~_i
    (i >= 1), so that the physical field is Re sum_i c_i e^{j omega_i t} (the
    one-sided form of the real two-sided series);
  * the a priori truncation error e_M^2 of Eq. mode_error for every candidate
    N_m: the squared relative L2(Gamma x T) distance between a field and its
    series truncated after mode N_m, summed over the fields given (Dirichlet
    g and, when present, Neumann h); the time integral is the rectangle rule
    on the same samples and the L2(Gamma) inner product a nodal quadrature
    with caller weights (unit weights: the nodal l2 norm);
  * the smallest N_m with e_M < epsilon_m (step 2 of the algorithm);
  * the a posteriori side of the same step: the L2(Omega x T) energy of every
    solved mode's velocity field Re(u~_k e^{j omega_k t}) and the relative
    change ||u^_N - u^_{N-1}||^2 / ||u^_N||^2 between the reconstructions
    (Eq. sol_reconstruct) truncated after modes N-1 and N, both evaluated
    literally from time samples of the reconstructions, the L2(Omega) norm
    with the P2 mass matrix M_s (as in Eq. total_error).
Each step follows the definition literally: coefficients by the sum, the
truncation error by reconstructing the truncated series at the samples.
"""
from __future__ import annotations

import numpy as np


def fourier_coefficients(g_t, n_modes):
    """g~_i, i = 0..n_modes-1, of real samples g_t [n_t][...] (Eq. SCVS_bc, rectangle rule)."""
    g_t = np.asarray(g_t, dtype=np.float64)
    n_t = g_t.shape[0]
    s = np.arange(n_t)
    out = np.empty((n_modes,) + g_t.shape[1:], dtype=np.complex128)
    for i in range(n_modes):
        e = np.exp(-2j * np.pi * i * s / n_t)
        out[i] = np.tensordot(e, g_t, axes=(0, 0)) / n_t
    return out


def solver_modes(coef):
    """Per-mode data of the solver: c_0 = g~_0, c_i = 2 g~_i for i >= 1."""
    c = np.array(coef, dtype=np.complex128, copy=True)
    c[1:] *= 2.0
    return c


def truncated_series(c, n_t, N):
    """Re sum_{i=0}^{N} c_i e^{j omega_i t_s} at the samples t_s = s T / n_t."""
    s = np.arange(n_t)
    out = np.zeros((n_t,) + c.shape[1:], dtype=np.float64)
    for i in range(N + 1):
        ph = np.exp(2j * np.pi * i * s / n_t)
        out += np.real(np.multiply.outer(ph, c[i]))
    return out


def _l2_gamma_t(f_t, w):
    """int_0^T ||f||^2_{L2(Gamma)} dt / T with the rectangle rule in time and nodal weights w
    (w broadcasts against the trailing axes of f_t)."""
    return float(np.mean(np.sum(w * f_t ** 2, axis=tuple(range(1, f_t.ndim)))))


def truncation_errors(fields, n_max):
    """e_M^2 of Eq. mode_error for N_m = 0..n_max-1.

    fields: list of (samples [n_t][...], weights broadcastable to [...]); the
    relative errors of the fields are added (the g and h terms of Eq.
    mode_error).  A field of zero norm contributes nothing."""
    e2 = np.zeros(n_max)
    for f_t, w in fields:
        f_t = np.asarray(f_t, dtype=np.float64)
        n_t = f_t.shape[0]
        if 2 * (n_max - 1) >= n_t:
            raise ValueError("modes must stay below the Nyquist frequency of the samples")
        norm2 = _l2_gamma_t(f_t, w)
        if norm2 == 0.0:
            continue
        c = solver_modes(fourier_coefficients(f_t, n_max))
        for N in range(n_max):
            e2[N] += _l2_gamma_t(f_t - truncated_series(c, n_t, N), w) / norm2
    return e2


def select_modes(fields, eps, n_max):
    """Smallest N_m with e_M < eps (None if no N_m < n_max reaches it)."""
    e2 = truncation_errors(fields, n_max)
    ok = np.flatnonzero(e2 < eps * eps)
    return (int(ok[0]) if ok.size else None), e2


def _l2_omega_t(Ms, u_t):
    """int_0^T ||u||^2_{L2(Omega)} dt / T of samples u_t [n_t][N][d] (rectangle rule; M_s per component)."""
    return float(np.mean([sum(u[:, c] @ (Ms @ u[:, c]) for c in range(u.shape[1])) for u in u_t]))


def _series(U, omegas, period, n_t, N):
    """Samples of Re sum_{k<=N} U_k e^{j omega_k t} (Eq. sol_reconstruct), [n_t][N][d]."""
    t = np.arange(n_t) * (period / n_t)
    out = np.zeros((n_t,) + U.shape[1:], dtype=np.float64)
    for s in range(n_t):
        acc = np.zeros(U.shape[1:], dtype=np.complex128)
        for k in range(N + 1):
            acc += U[k] * np.exp(1j * omegas[k] * t[s])
        out[s] = acc.real
    return out


def mode_energies(Ms, U, omegas, period, n_t):
    """E_k = mean over the period of ||Re(U_k e^{j omega_k t})||^2_{L2(Omega)}; U [m][N][d] complex."""
    out = np.zeros(len(omegas))
    t = np.arange(n_t) * (period / n_t)
    for k, w in enumerate(omegas):
        u_t = np.stack([np.real(U[k] * np.exp(1j * w * ts)) for ts in t])
        out[k] = _l2_omega_t(Ms, u_t)
    return out


def a_posteriori_increments(Ms, U, omegas, period, n_t):
    """delta_N^2 = ||u^_N - u^_{N-1}||^2 / ||u^_N||^2 in L2(Omega x T), N = 0..m-1 (u^_{-1} = 0;
    0 where ||u^_N|| = 0), from time samples of the two truncated reconstructions."""
    m = len(omegas)
    out = np.zeros(m)
    prev = np.zeros((n_t,) + U.shape[1:])
    for N in range(m):
        cur = _series(U, omegas, period, n_t, N)
        den = _l2_omega_t(Ms, cur)
        out[N] = _l2_omega_t(Ms, cur - prev) / den if den > 0 else 0.0
        prev = cur
    return out
