"""Pins of the Lanczos-DOS reference (Section 3.2.1): the quadrature of each
start vector reproduces its Chebyshev moments up to degree 2M-1 (Eq. tauexpand,
checked against the pinned KPM oracle), the weights sum to one, a diagonal
matrix with few distinct values is resolved exactly, and the blurred DOS with
M = n equals the blurred exact DOS."""
import numpy as np

from oracle import dos as odos
from oracle import kpm as okpm
from oracle import lanczos_dos as old
from synthetic import anderson_3d, diagonal, laplacian_2d


def test_quadrature_matches_kpm_moments_to_degree_2M_minus_1():
    A = anderson_3d(8, 5.0, seed=3)
    lb, ub = -9.0, 9.0
    c, d = 0.5 * (lb + ub), 0.5 * (ub - lb)
    M, nv = 12, 3
    mu = okpm.kpm_moments_per_vector(A, lb, ub, 2 * M - 1, nv, seed=4, mode="direct")
    for l, (theta, w) in enumerate(old.lanczos_ritz(A, M, nv, seed=4)):
        assert abs(w.sum() - 1.0) < 1e-12
        t = (theta - c) / d
        quad = np.array([np.sum(w * np.cos(k * np.arccos(np.clip(t, -1, 1)))) for k in range(2 * M)])
        assert np.abs(quad - mu[l]).max() < 1e-10


def test_few_distinct_values_resolved_exactly():
    vals = np.repeat([-1.0, 0.5, 3.0], [40, 25, 35])
    A = diagonal(vals)
    x = np.linspace(-3, 5, 801)
    phi = old.lanczos_dos(A, 10, 4, seed=2, sigma=0.2, x=x)
    V = okpm.start_block(A.n, 4, seed=2)
    exact = np.zeros_like(x)
    for l in range(4):
        w = V[:, l] ** 2 / A.n
        exact += (odos.gaussian(x[:, None] - vals[None, :], 0.2) * w[None, :]).sum(axis=1)
    exact /= 4
    assert np.abs(phi - exact).max() < 1e-10


def test_haydock_continued_fraction_full_run_is_lorentzian_of_spectrum():
    # With M = n the continued fraction is the exact resolvent entry, so the
    # Haydock DOS is the Lorentzian-blurred spectral measure of the vector.
    A = laplacian_2d(6)
    x = np.linspace(-1, 9, 401)
    eta = 0.25
    phi = old.haydock_dos(A, A.n, 1, seed=7, eta=eta, x=x)
    lam, U = np.linalg.eigh(A.to_dense())
    v = okpm.start_block(A.n, 1, seed=7)[:, 0]
    w = (U.T @ v) ** 2 / A.n
    ref = (w[None, :] * (eta / np.pi) / ((x[:, None] - lam[None, :]) ** 2 + eta ** 2)).sum(axis=1)
    assert np.abs(phi - ref).max() < 1e-9


def test_full_run_equals_blurred_exact_dos():
    A = laplacian_2d(6)                      # n = 36, distinct eigenvalues up to symmetry
    lam = np.linalg.eigvalsh(A.to_dense())
    x = np.linspace(-1, 9, 501)
    phi = old.lanczos_dos(A, A.n, 1, seed=5, sigma=0.3, x=x)
    # one vector: the blurred measure sum_j (u_j . v)^2 / n g(x - lambda_j)
    lam_all, U = np.linalg.eigh(A.to_dense())
    v = okpm.start_block(A.n, 1, seed=5)[:, 0]
    w = (U.T @ v) ** 2 / A.n
    ref = (odos.gaussian(x[:, None] - lam_all[None, :], 0.3) * w[None, :]).sum(axis=1)
    assert np.abs(phi - ref).max() < 1e-8
    del lam
