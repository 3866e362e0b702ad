"""Pins of the KPML / DGL reference (Section 3.1.3, Appendix B).

* Legendre moments from the vector recurrence equal sum_j w_j L_k(lambda_hat_j)
  with w_j = (u_j^T v)^2 / n from a dense eigendecomposition and L_k from
  scipy's Legendre evaluation; exact for a diagonal matrix; nu_0 = 1.
* The DGL coefficients from the recurrence of Eq. Leg3 equal the integral of
  Eq. DGLcoeff by high-order Gauss-Legendre quadrature (scipy's nodes).
* DGL with the exact Legendre moments reproduces the Gaussian-blurred exact DOS.
* KPML is the Legendre projection: its integrals against L_j return nu_j.
* Blurred KPML (quadrature) equals DGL without the stop test while the
  recurrence is converged -- two routes to <phi_L, g_sigma>.
"""
import math

import numpy as np
import pytest
import scipy.special

from oracle import dos as odos
from oracle import kpm as okpm
from oracle import legendre as oleg
from synthetic import anderson_3d, diagonal, laplacian_2d, random_symmetric


def _exact_weights(A, n_v, seed):
    lam, U = np.linalg.eigh(A.to_dense())
    V = okpm.start_block(A.n, n_v, seed)
    return lam, (U.T @ V) ** 2 / A.n          # (n, n_v)


@pytest.mark.parametrize("mat", ["random", "laplacian"])
def test_legendre_moments_match_dense_eig(mat):
    A = random_symmetric(120, 0.05, seed=8) if mat == "random" else laplacian_2d(9)
    lam, W = _exact_weights(A, 3, 11)
    lb, ub = lam.min() - 0.3, lam.max() + 0.2
    c, d = 0.5 * (lb + ub), 0.5 * (ub - lb)
    M = 60
    nu = oleg.legendre_moments_per_vector(A, lb, ub, M, 3, seed=11)
    Lk = np.array([scipy.special.eval_legendre(k, (lam - c) / d) for k in range(M + 1)])
    ref = (Lk @ W).T
    assert np.abs(nu - ref).max() < 1e-12
    assert np.abs(nu[:, 0] - 1.0).max() < 1e-14


def test_legendre_moments_diagonal_exact():
    vals = np.linspace(-2.0, 3.0, 57) ** 3 / 9.0
    A = diagonal(vals)
    lb, ub = -1.6, 3.2
    c, d = 0.5 * (lb + ub), 0.5 * (ub - lb)
    nu = oleg.legendre_moments(A, lb, ub, 40, 5, seed=3)
    ref = np.array([np.mean(scipy.special.eval_legendre(k, (vals - c) / d)) for k in range(41)])
    assert np.abs(nu - ref).max() < 1e-13
    assert np.all(np.abs(nu) <= 1.0 + 1e-14)


@pytest.mark.parametrize("t,sigma", [(0.0, 0.2), (0.55, 0.1), (-0.93, 0.05), (1.02, 0.08)])
def test_dgl_gamma_matches_quadrature_of_definition(t, sigma):
    # up to the paper's stop test (tol 1e-6) the recurrence is accurate to ~1e-11;
    # beyond it the recurrence amplifies its own rounding (Appendix B's warning)
    g = oleg.dgl_gamma(t, sigma, 400, tol=1e-6)
    s, w = scipy.special.roots_legendre(3000)
    G = np.exp(-0.5 * ((s - t) / sigma) ** 2)
    ref = np.array([np.sum(w * scipy.special.eval_legendre(k, s) * G) for k in range(g.shape[0])])
    assert g.shape[0] < 401                      # the stop test fired
    assert np.abs(g - ref).max() < 1e-10


def test_dgl_gamma_zero_order_closed_form():
    # gamma_0 = sigma sqrt(pi/2) [erf((1-t)/(sqrt2 sigma)) + erf((1+t)/(sqrt2 sigma))];
    # in the interior with a narrow Gaussian it tends to sigma sqrt(2 pi).
    assert abs(oleg.dgl_gamma(0.1, 0.01, 0)[0] - 0.01 * math.sqrt(2 * math.pi)) < 1e-15
    assert abs(oleg.dgl_gamma(1.0, 0.01, 0)[0] - 0.005 * math.sqrt(2 * math.pi)) < 1e-15


def test_stop_degree_grows_as_sigma_shrinks():
    used = [oleg.dgl_gamma(0.3, s, 5000).shape[0] - 1 for s in (0.4, 0.2, 0.1, 0.05)]
    assert used == sorted(used) and used[0] < used[-1] < 5000


def test_dgl_with_exact_moments_is_blurred_dos():
    A = anderson_3d(6, 5.0, seed=2)
    lam = np.linalg.eigvalsh(A.to_dense())
    lb, ub = lam.min() - 0.2, lam.max() + 0.2
    c, d = 0.5 * (lb + ub), 0.5 * (ub - lb)
    lh = (lam - c) / d
    M = 400
    nu = np.array([np.mean(scipy.special.eval_legendre(k, lh)) for k in range(M + 1)])
    sigma_t = 0.04
    t = np.linspace(-0.98, 0.98, 97)
    ref = odos.gaussian(t[:, None] - lh[None, :], sigma_t).mean(axis=1)
    # the stop test truncates the expansion: the error follows its tolerance
    for tol, bound in ((1e-6, 1e-3), (1e-8, 1e-5)):
        phi, used = oleg.dgl(nu, sigma_t, t, tol=tol)
        assert np.all(used < M)
        assert np.abs(phi - ref).max() < bound * ref.max()


def test_kpml_is_the_legendre_projection():
    A = random_symmetric(90, 0.06, seed=4)
    lam = np.linalg.eigvalsh(A.to_dense())
    lb, ub = lam.min() - 0.1, lam.max() + 0.1
    M = 25
    nu = oleg.legendre_moments(A, lb, ub, M, 4, seed=9)
    t, w = scipy.special.roots_legendre(M + 2)
    phi = oleg.kpml(nu, t)
    for j in range(M + 1):
        assert abs(np.sum(w * phi * scipy.special.eval_legendre(j, t)) - nu[j]) < 1e-12
    # the density integrates to nu_0 = 1 in t and in lambda
    x, wx = scipy.special.roots_legendre(M + 2)
    c, d = 0.5 * (lb + ub), 0.5 * (ub - lb)
    assert abs(np.sum(wx * d * oleg.kpml_lambda(nu, lb, ub, c + d * x)) - 1.0) < 1e-12


def test_blurred_kpml_equals_unstopped_dgl():
    A = laplacian_2d(8)
    lb, ub = -0.1, 8.1
    M = 12                                   # short enough for the recurrence to stay exact
    nu = oleg.legendre_moments(A, lb, ub, M, 6, seed=1)
    sigma = 0.6
    x = np.linspace(lb - 1.0, ub + 1.0, 301)
    a = oleg.blurred_kpml(nu, lb, ub, sigma, x, 400)
    b, used = oleg.dgl_lambda(nu, lb, ub, sigma, x, tol=0.0)
    assert np.all(used == M)
    assert np.abs(a - b).max() < 1e-11 * np.abs(a).max()


def test_legendre_error_zero_and_convergence():
    A = laplacian_2d(12)
    lam = np.linalg.eigvalsh(A.to_dense())
    lb, ub = -0.08, 8.08
    c, d = 0.5 * (lb + ub), 0.5 * (ub - lb)
    sigma = 0.35
    dgl, kpml = [], []
    for M in (20, 60, 160):
        nu = np.array([np.mean(scipy.special.eval_legendre(k, (lam - c) / d)) for k in range(M + 1)])
        dgl.append(oleg.legendre_error(nu, "dgl", lb, ub, sigma, eigs=lam)[0])
        kpml.append(oleg.legendre_error(nu, "kpml", lb, ub, sigma, eigs=lam)[0])
    # KPML converges to the blurred exact DOS; DGL until its stop test truncates
    assert kpml[0] > kpml[1] > kpml[2] and kpml[2] < 1e-10
    assert dgl[0] > dgl[1] >= dgl[2] and dgl[2] < 1e-4
