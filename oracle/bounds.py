"""Spectrum bounds (test infrastructure only).

Section 3.1 (around Eq. cd): the method needs lb <= lambda_min and
ub >= lambda_max before mapping A to B = (A - cI)/d.  Two ways:

* ``gershgorin`` -- the textbook disc bound (not in the paper; C code in
  kpm_oracle.c).
* ``lanczos``    -- the paper's suggestion: after a k-step Lanczos run
  (Eq. lanfact: A V_k = V_k T_k + f_k e_k^T), take
  ub = theta_max + ||(A - theta_max I) u||, lb = theta_min - ||(A - theta_min I) u||,
  where each residual norm equals ||f_k|| * |last entry of the Ritz vector of T_k|.

Both are widened by ``pad_frac * (ub - lb)`` on each side.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import scipy.linalg

from . import kpm


def gershgorin(A) -> tuple[float, float]:
    rp, ci, va = kpm._csr_arrays(A.row_ptr, A.col_idx, A.val)
    lo, hi = C.c_double(), C.c_double()
    kpm.lib().oracle_gershgorin(A.n, rp.ctypes.data, ci.ctypes.data, va.ctypes.data,
                                C.byref(lo), C.byref(hi))
    return lo.value, hi.value


def lanczos_tridiagonal(A, steps: int, seed: int, batch_index: int = 0):
    """Plain k-step Lanczos (no reorthogonalisation) from the normalised
    Rademacher start vector l = 0.  Returns (alpha[k], beta[k]) where beta[-1]
    is ||f_k||.  The run stops early at an invariant subspace, taken as
    beta_j <= 1e-12 * max_{i<=j}(|alpha_i| + beta_i + beta_{i-1}) (the paper is
    silent on breakdown)."""
    n = A.n
    q = kpm.start_block(n, 1, seed, batch_index)[:, 0]
    q = q / np.sqrt(q @ q)
    q_prev = np.zeros(n)
    beta_prev = 0.0
    alpha, beta = [], []
    scale = 0.0
    for j in range(min(steps, n)):
        w = kpm.spmv(A, q) - beta_prev * q_prev
        a = float(q @ w)
        w = w - a * q
        b = float(np.sqrt(w @ w))
        alpha.append(a)
        beta.append(b)
        scale = max(scale, abs(a) + b + beta_prev)
        if b <= 1e-12 * scale:
            break
        q_prev, q = q, w / b
        beta_prev = b
    return np.array(alpha), np.array(beta)


def lanczos(A, steps: int, seed: int, batch_index: int = 0) -> tuple[float, float]:
    alpha, beta = lanczos_tridiagonal(A, steps, seed, batch_index)
    theta, Y = scipy.linalg.eigh_tridiagonal(alpha, beta[:-1])
    f = beta[-1]
    lb = theta[0] - f * abs(Y[-1, 0])
    ub = theta[-1] + f * abs(Y[-1, -1])
    return float(lb), float(ub)


def pad(lb: float, ub: float, pad_frac: float) -> tuple[float, float]:
    w = ub - lb
    return lb - pad_frac * w, ub + pad_frac * w


def bounds(A, method: str = "gershgorin", steps: int = 20, seed: int = 0,
           pad_frac: float = 0.01) -> tuple[float, float]:
    if method == "gershgorin":
        lb, ub = gershgorin(A)
    elif method == "lanczos":
        lb, ub = lanczos(A, steps, seed)
    else:
        raise ValueError(method)
    return pad(lb, ub, pad_frac)
