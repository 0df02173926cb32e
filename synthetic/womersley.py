"""Analytic fully developed oscillatory flows (the paper's Sec. 3.2 channel
profile and Eq. Womersley_cmplx pipe profile), used to make Dirichlet inlet data and, in tests,
as the exact solution the oracle is pinned to.

Both are written per unit pressure-gradient amplitude G = h_x/L (the paper's
h_x/L, Sec. 3.2 and 3.4): the mode-k velocity is c_k * profile, the mode-k
pressure is c_k * G (L - x), which vanishes at the traction-free outlet.
"""
from __future__ import annotations

import numpy as np
import scipy.special as sps


def channel_profile(y, omega, half_height, rho, mu, G=1.0):
    """u_x(y) of plane oscillatory channel flow (Sec. 3.2).

    omega = 0: G/(2 mu) (H+y)(H-y);  omega != 0:
    -(j G/(rho omega)) [1 - cosh(Lam y/H)/cosh(Lam)],  Lam^2 = j W, W = omega H^2 rho/mu.
    The cosh ratio is evaluated in exponential form so that large W does
    not overflow.
    """
    y = np.asarray(y, dtype=np.float64)
    H = half_height
    if omega == 0.0:
        return (G / (2.0 * mu)) * (H + y) * (H - y) + 0j
    W = omega * H * H * rho / mu
    lam = np.sqrt(1j * W)  # principal root, Re > 0
    s = np.abs(y) / H
    ratio = np.exp(lam * (s - 1.0)) * (1.0 + np.exp(-2.0 * lam * s)) / (1.0 + np.exp(-2.0 * lam))
    return -(1j * G / (rho * omega)) * (1.0 - ratio)


def pipe_profile(r, omega, radius, rho, mu, G=1.0):
    """u_x(r) of Womersley pipe flow (Eq. Womersley_cmplx).

    omega = 0: G/(4 mu)(R^2 - r^2);  omega != 0:
    -(j G/(rho omega)) [1 - J0(Lam r/R)/J0(Lam)],  Lam^2 = -j W, W = omega R^2 rho/mu.
    """
    r = np.asarray(r, dtype=np.float64)
    R = radius
    if omega == 0.0:
        return (G / (4.0 * mu)) * (R * R - r * r) + 0j
    W = omega * R * R * rho / mu
    lam = np.sqrt(-1j * W)
    return -(1j * G / (rho * omega)) * (1.0 - sps.jv(0, lam * r / R) / sps.jv(0, lam))
