"""Reconstruction and accuracy metric (test infrastructure only).

* Jackson damping factors g_k^M (Appendix A, Eq. jackson), alpha_M = pi/(M+2).
* Truncated expansion (Eq. tdosFinal) with the paper's coefficients
  (2 - delta_k0)/pi (Eq. expmu) applied to moments normalised so mu_0 = 1:
      phi_hat(t) = [g_0 mu_0 + 2 sum_{k>=1} g_k mu_k T_k(t)] / (pi sqrt(1 - t^2)),
  and in eigenvalue units phi(lambda) = phi_hat((lambda - c)/d) / d.
  T_k(t) is evaluated from its closed form cos(k arccos t).
* Gaussian test function g_sigma (Eq. gauss) and the regularised DOS
  phi_sigma(x) = (1/n) sum_j g_sigma(x - lambda_j) (Eq. blurphi, with the 1/n of
  Eq. DOS0 restored so that it integrates to one).
* The KPM approximation is blurred the same way, <phi_tilde, g_sigma(. - x)>
  (Section 4), by Gauss-Chebyshev quadrature on N_q nodes:
      (1/N_q) sum_i P(t_i) g_sigma(x - c - d t_i),  t_i = cos(pi (i + 1/2) / N_q),
  with P(t) the bracket above; N_q = max(4 (M+1), ceil(40 d / sigma)).
* Errors (Eq. err2 with p = 1, and the sup-norm of Eq. errormetric) on a
  uniform grid of N_x points over [lb - 6 sigma, ub + 6 sigma]; the L1 norm by
  the trapezoid rule.
"""
from __future__ import annotations

import math

import numpy as np


def jackson(M: int) -> np.ndarray:
    a = math.pi / (M + 2)
    k = np.arange(M + 1, dtype=np.float64)
    return ((1.0 - k / (M + 2)) * math.sin(a) * np.cos(k * a)
            + (1.0 / (M + 2)) * math.cos(a) * np.sin(k * a)) / math.sin(a)


def damping_factors(M: int, damping: str) -> np.ndarray:
    if damping == "jackson":
        return jackson(M)
    if damping == "none":
        return np.ones(M + 1)
    raise ValueError(damping)


def chebyshev_nodes(N: int) -> np.ndarray:
    """Ascending Chebyshev nodes t_i = -cos(pi (i + 1/2) / N)."""
    return -np.cos(np.pi * (np.arange(N) + 0.5) / N)


def _poly(mu: np.ndarray, g: np.ndarray, t: np.ndarray) -> np.ndarray:
    """P(t) = g_0 mu_0 + 2 sum_{k>=1} g_k mu_k T_k(t), T_k(t) = cos(k arccos t)."""
    M = mu.shape[0] - 1
    k = np.arange(M + 1)
    T = np.cos(np.outer(np.arccos(np.clip(t, -1.0, 1.0)), k))
    coef = g * mu * np.where(k == 0, 1.0, 2.0)
    return T @ coef


def reconstruct(mu, damping: str = "jackson", t=None, N_t: int = 1000,
                lb: float | None = None, ub: float | None = None):
    """phi_hat on the t-grid (default: N_t ascending Chebyshev nodes).

    Returns (t, phi_hat, phi_lambda) with phi_lambda None unless lb, ub given."""
    mu = np.asarray(mu, dtype=np.float64)
    M = mu.shape[0] - 1
    t = chebyshev_nodes(N_t) if t is None else np.asarray(t, dtype=np.float64)
    g = damping_factors(M, damping)
    phi_hat = _poly(mu, g, t) / (np.pi * np.sqrt(1.0 - t * t))
    phi_lambda = None
    if lb is not None and ub is not None:
        d = 0.5 * (ub - lb)
        phi_lambda = phi_hat / d
    return t, phi_hat, phi_lambda


def gaussian(x, sigma):
    return np.exp(-0.5 * (x / sigma) ** 2) / math.sqrt(2.0 * math.pi * sigma * sigma)


def x_grid(lb: float, ub: float, sigma: float, N_x: int = 4000) -> np.ndarray:
    return np.linspace(lb - 6.0 * sigma, ub + 6.0 * sigma, N_x)


def quadrature_nodes(M: int, lb: float, ub: float, sigma: float) -> int:
    d = 0.5 * (ub - lb)
    return max(4 * (M + 1), int(math.ceil(40.0 * d / sigma)))


def blurred_kpm(mu, damping, lb, ub, sigma, x, N_q: int) -> np.ndarray:
    mu = np.asarray(mu, dtype=np.float64)
    M = mu.shape[0] - 1
    c, d = 0.5 * (lb + ub), 0.5 * (ub - lb)
    t = np.cos(np.pi * (np.arange(N_q) + 0.5) / N_q)
    P = _poly(mu, damping_factors(M, damping), t)
    G = gaussian(x[:, None] - c - d * t[None, :], sigma)
    return (G @ P) / N_q


def blurred_exact(eigs, sigma, x) -> np.ndarray:
    eigs = np.asarray(eigs, dtype=np.float64)
    out = np.zeros_like(x)
    for s in range(0, eigs.shape[0], 2048):
        out += gaussian(x[:, None] - eigs[None, s:s + 2048], sigma).sum(axis=1)
    return out / eigs.shape[0]


def smoothed_error(mu, damping: str, lb: float, ub: float, sigma: float, *,
                   eigs=None, ref_mu=None, ref_damping: str = "jackson",
                   N_x: int = 4000) -> tuple[float, float]:
    """(E_1, E_inf) between the blurred KPM DOS and the blurred reference."""
    mu = np.asarray(mu, dtype=np.float64)
    x = x_grid(lb, ub, sigma, N_x)
    M_eff = mu.shape[0] - 1
    if ref_mu is not None:
        M_eff = max(M_eff, len(ref_mu) - 1)
    N_q = quadrature_nodes(M_eff, lb, ub, sigma)
    approx = blurred_kpm(mu, damping, lb, ub, sigma, x, N_q)
    if eigs is not None:
        ref = blurred_exact(eigs, sigma, x)
    elif ref_mu is not None:
        ref = blurred_kpm(ref_mu, ref_damping, lb, ub, sigma, x, N_q)
    else:
        raise ValueError("need eigs or ref_mu")
    diff = np.abs(approx - ref)
    h = x[1] - x[0]
    e1 = h * (diff.sum() - 0.5 * (diff[0] + diff[-1]))
    return float(e1), float(diff.max())
