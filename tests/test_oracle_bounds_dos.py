"""Pins of the oracle's bounds, reconstruction and error metric.

Bounds (Section 3.1): Gershgorin is checked on matrices whose disc bound is
known in closed form and against dense spectra; the Lanczos bound against the
exact spectrum when the run spans the whole space.  Reconstruction (Eq.
tdosFinal, Appendix A Jackson damping) is checked through Chebyshev
orthogonality by Gauss-Chebyshev quadrature, non-negativity of the damped
kernel (Section 4) and the Jackson endpoint g_{M+1} = 0.  The metric (Eqs.
gauss, blurphi, err2, errormetric) through normalisation, the zero of
identical inputs and convergence to the exactly blurred spectrum.
"""
import math

import numpy as np
import pytest

from oracle import bounds, dos, kpm
from synthetic import anderson_3d, diagonal, laplacian_2d, random_symmetric


def test_gershgorin_laplacian_and_diagonal():
    lb, ub = bounds.gershgorin(laplacian_2d(40))
    assert (lb, ub) == (0.0, 8.0)     # interior rows: 4 +- 4
    d = np.array([3.0, -1.5, 2.25, 0.0])
    assert bounds.gershgorin(diagonal(d)) == (-1.5, 3.0)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_gershgorin_encloses_spectrum(seed):
    A = random_symmetric(80, 0.08, seed, empty_rows=3)
    lam = np.linalg.eigvalsh(A.to_dense())
    lb, ub = bounds.gershgorin(A)
    assert lb <= lam[0] + 1e-12 and ub >= lam[-1] - 1e-12


def test_lanczos_full_run_recovers_extremes():
    # With k = n distinct eigenvalues the Ritz values are the eigenvalues and the
    # residual vanishes, so the bounds are the exact extremes.
    rng = np.random.default_rng(4)
    dvals = np.sort(rng.uniform(-2.0, 3.0, size=24))
    A = diagonal(dvals)
    alpha, beta = bounds.lanczos_tridiagonal(A, 24, seed=0)
    T = np.diag(alpha) + np.diag(beta[:-1], 1) + np.diag(beta[:-1], -1)
    assert np.allclose(np.linalg.eigvalsh(T), dvals, atol=1e-9)
    lb, ub = bounds.lanczos(A, 24, seed=0)
    assert abs(lb - dvals[0]) < 1e-8 and abs(ub - dvals[-1]) < 1e-8


def test_lanczos_stops_at_invariant_subspace():
    # Three distinct eigenvalues: the Krylov space of any start vector has
    # dimension 3, so the run ends after 3 steps with the exact extremes.
    A = diagonal(np.repeat([1.0, 2.0, 4.0], 50))
    alpha, beta = bounds.lanczos_tridiagonal(A, 20, seed=0)
    assert len(alpha) == 3 and beta[-1] < 1e-12
    lb, ub = bounds.lanczos(A, 20, seed=0)
    assert abs(lb - 1.0) < 1e-12 and abs(ub - 4.0) < 1e-12


def test_lanczos_20_steps_bracket_laplacian():
    m = 40
    i = np.arange(1, m + 1)
    lam = (4 - 2 * np.cos(i[:, None] * np.pi / (m + 1)) - 2 * np.cos(i[None, :] * np.pi / (m + 1)))
    lb, ub = bounds.bounds(laplacian_2d(m), "lanczos", steps=20, seed=0, pad_frac=0.01)
    assert lb <= lam.min() and ub >= lam.max()
    # Ritz values move inward from the true extremes; the residual term widens them.
    lb0, ub0 = bounds.lanczos(laplacian_2d(m), 20, seed=0)
    assert ub0 > 7.5 and lb0 < 0.5


def test_lanczos_anderson_encloses():
    A = anderson_3d(10, 4.0, seed=1)
    lam = np.linalg.eigvalsh(A.to_dense())
    lb, ub = bounds.bounds(A, "lanczos", steps=30, seed=3, pad_frac=0.01)
    assert lb <= lam[0] and ub >= lam[-1]


def test_jackson_factors():
    for M in (0, 1, 10, 100, 257):
        g = dos.jackson(M)
        assert g.shape == (M + 1,)
        assert abs(g[0] - 1.0) < 1e-15
        assert np.all(np.diff(g) < 0)                  # a low-pass factor, decreasing in k
        assert np.all(g > 0)
        # The formula continued to k = M+1 vanishes: the kernel has degree M.
        a = math.pi / (M + 2)
        k = M + 1
        gk = ((1 - k / (M + 2)) * math.sin(a) * math.cos(k * a)
              + math.cos(a) * math.sin(k * a) / (M + 2)) / math.sin(a)
        assert abs(gk) < 1e-13


@pytest.mark.parametrize("damping", ["none", "jackson"])
def test_reconstruction_chebyshev_orthogonality(damping):
    # (pi/N) sum_i sqrt(1 - t_i^2) phi_hat(t_i) T_j(t_i) = g_j mu_j (j >= 1) and
    # g_0 mu_0 (j = 0): Gauss-Chebyshev is exact below degree 2N.
    rng = np.random.default_rng(1)
    M = 60
    mu = np.concatenate([[1.0], rng.uniform(-0.5, 0.5, M)])
    g = dos.damping_factors(M, damping)
    N = 400
    t, phi, _ = dos.reconstruct(mu, damping, N_t=N)
    assert np.all(np.diff(t) > 0)
    w = np.pi / N * np.sqrt(1 - t * t) * phi
    for j in range(M + 1):
        val = np.sum(w * np.cos(j * np.arccos(t)))
        assert abs(val - g[j] * mu[j]) < 1e-12


def test_damped_kernel_nonnegative_and_undamped_gibbs():
    # A spectrum concentrated at one point gives mu_k = T_k(t0): the damped
    # expansion is the Jackson kernel, which is non-negative; the plain
    # truncation oscillates below zero (Gibbs).
    M = 40
    t0 = 0.3
    mu = np.cos(np.arange(M + 1) * np.arccos(t0))
    t = np.linspace(-0.999, 0.999, 2001)
    _, pj, _ = dos.reconstruct(mu, "jackson", t=t)
    _, pn, _ = dos.reconstruct(mu, "none", t=t)
    assert pj.min() >= -1e-12 * pj.max()
    assert pn.min() < -0.05 * pn.max()


def test_damped_dos_nonnegative_for_stochastic_moments():
    A = laplacian_2d(40)
    mu = kpm.kpm_moments(A, -0.08, 8.08, 100, 20, seed=1)
    _, phi, _ = dos.reconstruct(mu, "jackson", N_t=1000)
    assert phi.min() >= -1e-12 * phi.max()
    # integrates to mu_0 = 1 by Gauss-Chebyshev on the default grid
    t = dos.chebyshev_nodes(1000)
    assert abs(np.pi / 1000 * np.sum(np.sqrt(1 - t * t) * phi) - 1.0) < 1e-12


def test_gaussian_and_blurred_exact_normalised():
    x = np.linspace(-5, 5, 20001)
    assert abs(np.trapezoid(dos.gaussian(x, 0.35), x) - 1.0) < 1e-12
    lam = np.random.default_rng(0).uniform(0, 8, 500)
    xg = dos.x_grid(0.0, 8.0, 0.35)
    assert abs(np.trapezoid(dos.blurred_exact(lam, 0.35, xg), xg) - 1.0) < 1e-9


def test_smoothed_error_zero_and_convergence():
    m = 40
    i = np.arange(1, m + 1)
    lam = (4 - 2 * np.cos(i[:, None] * np.pi / (m + 1))
           - 2 * np.cos(i[None, :] * np.pi / (m + 1))).ravel()
    lb, ub = -0.08, 8.08
    c, d = 0.5 * (lb + ub), 0.5 * (ub - lb)
    sigma = 0.35

    def exact_mu(M):
        return np.array([np.mean(np.cos(k * np.arccos((lam - c) / d))) for k in range(M + 1)])

    mu = exact_mu(80)
    e1, einf = dos.smoothed_error(mu, "jackson", lb, ub, sigma, ref_mu=mu)
    assert e1 == 0.0 and einf == 0.0
    errs = [dos.smoothed_error(exact_mu(M), "jackson", lb, ub, sigma, eigs=lam)[0]
            for M in (10, 20, 40, 80, 160)]
    assert all(a > b for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-2
    # blurred KPM with exact moments converges to the blurred exact DOS pointwise
    x = dos.x_grid(lb, ub, sigma)
    approx = dos.blurred_kpm(exact_mu(400), "none", lb, ub, sigma, x,
                             dos.quadrature_nodes(400, lb, ub, sigma))
    assert np.abs(approx - dos.blurred_exact(lam, sigma, x)).max() < 1e-6
