"""KPML and the Delta-Gauss-Legendre (DGL) method -- test infrastructure only.

Section 3.1.1 names KPML (the KPM expansion with Legendre instead of Chebyshev
polynomials); Section 3.1.3 and Appendix B derive DGL (Eq. DGLexp, DGLcoeff,
dglexpansion, gam0, eta, Leg3, StopRecur; Algorithm DGL).

* Legendre moments, B = (A - cI)/d:
      nu_k = (1/(n n_v)) sum_l v_l^T L_k(B) v_l,
  from the vector recurrence of Algorithm DGL, v_1 = B v_0,
  v_{k+1} = ((2k+1) B v_k - k v_{k-1}) / (k+1), and the direct dots v_0^T v_k
  (C oracle, mode "legendre").  Rademacher start vectors, so the paper's
  "normalized v_0" becomes the 1/n.
* KPML density in t (undamped; the paper gives no damping for Legendre):
      phi_L(t) = sum_{k=0}^{M} (k + 1/2) nu_k L_k(t),
  with L_k from the three-term recurrence (k+1) L_{k+1} = (2k+1) t L_k - k L_{k-1}.
* DGL coefficients gamma_k(t) = int_{-1}^{1} L_k(s) exp(-((s - t)/sigma)^2 / 2) ds
  from gamma_0 (Eq. gam0, erf) and the joint recurrence of Eq. Leg3 with
  psi_0 = 0, psi_1 = gamma_0 and zeta_k of Eq. eta, stopped by Eq. StopRecur
  (|gamma_{k-1}| + |gamma_k| <= k tol, absolute tol, 1e-6 by default) or at M.
  The DGL density at t is (2 pi sigma^2)^{-1/2} sum_{k<=M_t} (k + 1/2) gamma_k(t) nu_k.
* In eigenvalue units a density in t maps as phi(lambda) = phi_t((lambda - c)/d) / d,
  and a width sigma in lambda is sigma / d in t.
* Blurred KPML (for the error metric of Section 4): <phi_L, g_sigma(. - x)> by
  Gauss-Legendre quadrature in t on N_q nodes (scipy's nodes and weights),
  N_q = max(4 (M + 1), ceil(40 d / sigma)) as for KPM.  DGL is already a
  Gaussian-regularised density and is compared directly.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.special

from . import dos as odos
from . import kpm


def legendre_moments_per_vector(A, lb: float, ub: float, M: int, n_v: int, seed: int,
                                **kw) -> np.ndarray:
    """nu_k^(l) = v_l^T L_k(B) v_l / n, shape (n_v, M+1)."""
    return kpm.kpm_moments_per_vector(A, lb, ub, M, n_v, seed, mode="legendre", **kw)


def legendre_moments(A, lb, ub, M, n_v, seed, **kw) -> np.ndarray:
    return legendre_moments_per_vector(A, lb, ub, M, n_v, seed, **kw).mean(axis=0)


def legendre_values(M: int, t) -> np.ndarray:
    """L_0..L_M at the points t, shape (M+1, len(t))."""
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    L = np.empty((M + 1, t.shape[0]))
    L[0] = 1.0
    if M >= 1:
        L[1] = t
    for k in range(1, M):
        L[k + 1] = ((2 * k + 1) * t * L[k] - k * L[k - 1]) / (k + 1)
    return L


def kpml(nu, t) -> np.ndarray:
    """phi_L(t) = sum_k (k + 1/2) nu_k L_k(t)."""
    nu = np.asarray(nu, dtype=np.float64)
    M = nu.shape[0] - 1
    L = legendre_values(M, t)
    return ((np.arange(M + 1) + 0.5) * nu) @ L


def kpml_lambda(nu, lb: float, ub: float, x) -> np.ndarray:
    c, d = 0.5 * (lb + ub), 0.5 * (ub - lb)
    return kpml(nu, (np.asarray(x, dtype=np.float64) - c) / d) / d


def dgl_gamma(t: float, sigma: float, M: int, tol: float = 1e-6) -> np.ndarray:
    """gamma_0..gamma_{M_t} at one point t (sigma in t units); tol <= 0 never stops early."""
    s2 = sigma * sigma
    r = math.sqrt(2.0) * sigma
    g0 = sigma * math.sqrt(math.pi / 2.0) * (math.erf((1.0 - t) / r) + math.erf((1.0 + t) / r))
    e_plus = math.exp(-0.5 * ((1.0 - t) / sigma) ** 2)
    e_minus = math.exp(-0.5 * ((1.0 + t) / sigma) ** 2)
    gam = [g0]
    g_prev, g_cur = 0.0, g0           # gamma_{k-1}, gamma_k
    p_prev, p_cur = 0.0, 0.0          # psi_{k-1}, psi_k
    for k in range(M):
        zeta = e_plus - (e_minus if k % 2 == 0 else -e_minus)
        g_next = ((2 * k + 1) * (s2 * (p_cur - zeta) + t * g_cur) - k * g_prev) / (k + 1)
        p_next = (2 * k + 1) * g_cur + p_prev
        gam.append(g_next)
        g_prev, g_cur = g_cur, g_next
        p_prev, p_cur = p_cur, p_next
        kk = k + 1
        if tol > 0.0 and abs(g_prev) + abs(g_cur) <= kk * tol:
            break
    return np.array(gam)


def dgl(nu, sigma: float, t, tol: float = 1e-6):
    """(phi(t_i), M_i) for the points t_i; sigma in t units."""
    nu = np.asarray(nu, dtype=np.float64)
    M = nu.shape[0] - 1
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    phi = np.empty(t.shape[0])
    used = np.empty(t.shape[0], dtype=np.int64)
    pref = 1.0 / math.sqrt(2.0 * math.pi * sigma * sigma)
    for i, ti in enumerate(t):
        g = dgl_gamma(float(ti), sigma, M, tol)
        k = np.arange(g.shape[0])
        phi[i] = pref * np.sum((k + 0.5) * g * nu[:g.shape[0]])
        used[i] = g.shape[0] - 1
    return phi, used


def dgl_lambda(nu, lb: float, ub: float, sigma: float, x, tol: float = 1e-6):
    c, d = 0.5 * (lb + ub), 0.5 * (ub - lb)
    phi, used = dgl(nu, sigma / d, (np.asarray(x, dtype=np.float64) - c) / d, tol)
    return phi / d, used


def blurred_kpml(nu, lb: float, ub: float, sigma: float, x, N_q: int) -> np.ndarray:
    c, d = 0.5 * (lb + ub), 0.5 * (ub - lb)
    t, w = scipy.special.roots_legendre(N_q)
    P = kpml(nu, t)
    G = odos.gaussian(np.asarray(x)[:, None] - c - d * t[None, :], sigma)
    return G @ (w * P)


def legendre_error(nu, method: str, lb: float, ub: float, sigma: float, *, eigs=None,
                   ref_mu=None, ref_damping: str = "jackson", tol: float = 1e-6,
                   N_x: int = 4000) -> tuple[float, float]:
    """(E_1, E_inf) of KPML ("kpml", blurred) or DGL ("dgl") against the blurred
    exact DOS (eigs) or a blurred Chebyshev reference (ref_mu), on the grid and
    with the trapezoid rule of the KPM metric."""
    nu = np.asarray(nu, dtype=np.float64)
    M = nu.shape[0] - 1
    x = odos.x_grid(lb, ub, sigma, N_x)
    M_eff = M if ref_mu is None else max(M, len(ref_mu) - 1)
    N_q = odos.quadrature_nodes(M_eff, lb, ub, sigma)
    if method == "kpml":
        approx = blurred_kpml(nu, lb, ub, sigma, x, N_q)
    elif method == "dgl":
        approx = dgl_lambda(nu, lb, ub, sigma, x, tol)[0]
    else:
        raise ValueError("method must be 'kpml' or 'dgl'")
    if eigs is not None:
        ref = odos.blurred_exact(eigs, sigma, x)
    elif ref_mu is not None:
        ref = odos.blurred_kpm(ref_mu, ref_damping, lb, ub, sigma, x, N_q)
    else:
        raise ValueError("need eigs or ref_mu")
    diff = np.abs(approx - ref)
    h = x[1] - x[0]
    e1 = h * (diff.sum() - 0.5 * (diff[0] + diff[-1]))
    return float(e1), float(diff.max())
