"""Lanczos DOS with Gaussian-blurred Ritz values (Section 3.2.1, Eq. landos) --
test infrastructure only.

For each start vector v_l (the same Rademacher vectors as the KPM sweep,
normalised to unit length), an M-step Lanczos run (Eq. lanfact, plain
three-term recurrence, no reorthogonalisation) gives the tridiagonal T_M; its
eigenvalues theta_k (Ritz values) and the squared first components tau_k^2 of
its unit eigenvectors form a quadrature for the vector's spectral measure
(Eq. landist, Eq. tauexpand).  The approximate DOS is

    phi_sigma(t) = (1/n_v) sum_l sum_k tau_{k,l}^2 g_sigma(t - theta_{k,l}).

Reading: the paper writes an extra 1/n in front of the inner sum; with unit
start vectors the weights of each vector already sum to one, so the 1/n
belongs to unnormalised vectors (|v|^2 = n) and is dropped here so that the
DOS integrates to one (as Eq. avgphi does).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from . import kpm
from .dos import gaussian


def lanczos_run(A, q0: np.ndarray, M: int):
    """M steps from unit vector q0: (alpha[m], beta[m]) with beta[m-1] = ||f_m||;
    stops early (m < M) when beta_j <= 1e-12 * running norm estimate."""
    q = q0 / np.sqrt(q0 @ q0)
    q_prev = np.zeros_like(q)
    beta_prev = 0.0
    alpha, beta = [], []
    scale = 0.0
    for _ in range(M):
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


def ritz(alpha: np.ndarray, beta: np.ndarray):
    """Ritz values and squared first eigenvector components of T."""
    theta, Y = scipy.linalg.eigh_tridiagonal(alpha, beta[:-1])
    return theta, Y[0, :] ** 2


def lanczos_ritz(A, M: int, n_v: int, seed: int, batch_index: int = 0, vec_offset: int = 0):
    """Per start vector: list of (theta, tau^2)."""
    V = kpm.start_block(A.n, n_v, seed, batch_index, vec_offset)
    out = []
    for l in range(n_v):
        a, b = lanczos_run(A, V[:, l], M)
        out.append(ritz(a, b))
    return out


def haydock_dos(A, M: int, n_v: int, seed: int, eta: float, x: np.ndarray, **kw) -> np.ndarray:
    """Haydock's method (Section 3.2.2): -(1/pi) Im of the continued fraction
    e_1^T ((x + i eta) - T_M)^{-1} e_1, evaluated from the bottom up
    (G_{m+1} = 0, G_j = 1 / (z - alpha_j - beta_j^2 G_{j+1})), averaged over the
    unit start vectors."""
    V = kpm.start_block(A.n, n_v, seed, kw.get("batch_index", 0), kw.get("vec_offset", 0))
    z = np.asarray(x, dtype=np.float64) + 1j * eta
    acc = np.zeros(z.shape[0])
    for l in range(n_v):
        a, b = lanczos_run(A, V[:, l], M)
        G = np.zeros_like(z)
        for j in range(len(a) - 1, -1, -1):
            b2 = b[j] ** 2 if j < len(a) - 1 else 0.0
            G = 1.0 / (z - a[j] - b2 * G)
        acc += -G.imag / np.pi
    return acc / n_v


def lanczos_dos(A, M: int, n_v: int, seed: int, sigma: float, x: np.ndarray, **kw) -> np.ndarray:
    """Eq. landos on the points x."""
    acc = np.zeros_like(np.asarray(x, dtype=np.float64))
    for theta, w in lanczos_ritz(A, M, n_v, seed, **kw):
        acc += (gaussian(x[:, None] - theta[None, :], sigma) * w[None, :]).sum(axis=1)
    return acc / n_v
