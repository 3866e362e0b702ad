"""Pins of the heat-capacity reference (Section 4.3): the kernel's series at
small x and its limit 1 at infinite temperature, the Gauss-Chebyshev integral
of exact moments converging to the exact (1/n) sum_j g(lambda_j), and the
Jackson-damped estimate's error decreasing with M."""
import numpy as np

from oracle import observables as obs


def test_kernel_series_and_limits():
    x = np.array([1e-3, 1e-2, 0.1])
    # (y / sinh y)^2 with y = x/2: 1 - x^2/12 + x^4/240 - x^6/6048 + ...
    series = 1 - x ** 2 / 12 + x ** 4 / 240 - x ** 6 / 6048
    assert np.allclose(obs.heat_kernel(x ** 2, 1.0), series, rtol=0, atol=1e-12)
    assert obs.heat_kernel(0.0, 5.0) == 1.0
    assert obs.heat_kernel(4.0, 100.0) < 1e-80


def test_kpm_quadrature_converges_to_exact():
    m = 30
    i = np.arange(1, m + 1)
    lam = (4 - 2 * np.cos(i[:, None] * np.pi / (m + 1)) - 2 * np.cos(i[None, :] * np.pi / (m + 1))).ravel()
    lb, ub = -0.08, 8.08
    c, d = 0.5 * (lb + ub), 0.5 * (ub - lb)
    betas = np.array([0.3, 1.0, 3.0])
    exact = obs.heat_capacity_points(lam, np.ones_like(lam), betas)

    def mu_exact(M):
        t = (lam - c) / d
        return np.array([np.mean(np.cos(k * np.arccos(t))) for k in range(M + 1)])
    errs = [np.abs(obs.heat_capacity_kpm(mu_exact(M), "jackson", lb, ub, betas) - exact).max()
            for M in (10, 40, 160)]
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-3
    undamped = obs.heat_capacity_kpm(mu_exact(600), "none", lb, ub, betas)
    assert np.abs(undamped - exact).max() < 1e-4
