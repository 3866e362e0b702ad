"""An observable of the DOS: the heat capacity of Section 4.3 -- test
infrastructure only.

C_v(T) = <phi, g> with g of Eq. gfunc up to its constant factor,
    g(lambda) = x^2 e^{-x} / (1 - e^{-x})^2,   x = beta sqrt(max(lambda, 0)),
beta = hbar c / (k_B T).  The error of an estimate is Eq. errormetric_g.
"""
from __future__ import annotations

import numpy as np

from .dos import _poly, damping_factors


def heat_kernel(lam, beta):
    x = beta * np.sqrt(np.maximum(np.asarray(lam, dtype=np.float64), 0.0))
    small = x < 1e-6
    xs = np.where(small, 1.0, x)
    val = xs * xs * np.exp(-xs) / np.expm1(-xs) ** 2
    return np.where(small, 1.0 - x * x / 12.0, val)


def heat_capacity_points(pts, wts, betas):
    pts = np.asarray(pts, dtype=np.float64).ravel()
    wts = np.asarray(wts, dtype=np.float64).ravel()
    return np.array([np.sum(wts * heat_kernel(pts, b)) / wts.sum() for b in betas])


def heat_capacity_kpm(mu, damping, lb, ub, betas, N_q=None):
    """(1/N_q) sum_i P(t_i) g(c + d t_i), t_i = cos(pi (i + 1/2)/N_q)."""
    mu = np.asarray(mu, dtype=np.float64)
    M = mu.shape[0] - 1
    N_q = N_q or max(4 * (M + 1), 2048)
    c, d = 0.5 * (lb + ub), 0.5 * (ub - lb)
    t = np.cos(np.pi * (np.arange(N_q) + 0.5) / N_q)
    P = _poly(mu, damping_factors(M, damping), t)
    return np.array([np.sum(P * heat_kernel(c + d * t, b)) / N_q for b in betas])
