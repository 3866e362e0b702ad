"""The Lanczos DOS on the GPU (Section 3.2.1) against the oracle: tridiagonal
coefficients for short runs, the Gauss quadrature reproducing the Chebyshev
moments to degree 2M-1 (a property that does not depend on the rounding order
of long runs), the blurred DOS, and the points error metric."""
import numpy as np
import pytest

from oracle import dos as odos
from oracle import kpm as okpm
from oracle import lanczos_dos as old
from synthetic import anderson_3d, diagonal, laplacian_2d

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1308_5467_gb300 import dos
    c = dos.Context(0)
    yield c
    c.close()


def dev(A):
    from paper_1308_5467_gb300 import dos
    return dos.CSRArrays.from_synthetic(A, device="cuda")


@pytest.mark.parametrize("n_v", [1, 3, 16, 64])
def test_short_runs_match_oracle(ctx, n_v):
    A = anderson_3d(9, 5.0, seed=1)
    M = 12
    theta, weight, m_used = ctx.dos_lanczos_ritz(dev(A), M, n_v, seed=2)
    ref = old.lanczos_ritz(A, M, n_v, seed=2)
    for l in range(n_v):
        rt, rw = ref[l]
        assert m_used[l] == M
        assert np.abs(np.sort(theta[l]) - rt).max() < 1e-9
        order = np.argsort(theta[l])
        assert np.abs(weight[l][order] - rw).max() < 1e-9
        assert abs(weight[l].sum() - 1.0) < 1e-12


def test_quadrature_reproduces_moments(ctx):
    A = anderson_3d(12, 4.0, seed=3)
    lb, ub = -8.2, 8.2
    c, d = 0.5 * (lb + ub), 0.5 * (ub - lb)
    M, n_v = 60, 8
    theta, weight, _ = ctx.dos_lanczos_ritz(dev(A), M, n_v, seed=5)
    mu = okpm.kpm_moments_per_vector(A, lb, ub, 2 * M - 1, n_v, seed=5)
    for l in range(n_v):
        t = (theta[l] - c) / d
        quad = np.array([np.sum(weight[l] * np.cos(k * np.arccos(np.clip(t, -1, 1))))
                         for k in range(2 * M)])
        assert np.abs(quad - mu[l]).max() < 1e-8


def test_invariant_subspace_and_dos(ctx):
    vals = np.repeat([-1.0, 0.5, 3.0], [40, 25, 35])
    A = diagonal(vals)
    theta, weight, m_used = ctx.dos_lanczos_ritz(dev(A), 10, 4, seed=2)
    assert np.all(m_used == 3)
    x = np.linspace(-3, 5, 801)
    phi = ctx.dos_lanczos_dos(theta, weight, 0.2, x)
    ref = old.lanczos_dos(A, 10, 4, seed=2, sigma=0.2, x=x)
    assert np.abs(phi - ref).max() < 1e-10


def test_long_runs_with_ghost_copies(ctx):
    """M = 300 steps on the 900-row Laplacian: loss of orthogonality makes copies of
    converged Ritz values (they are merged into one node per group).  Weights are
    non-negative and sum to one, the Ritz values are ascending, and the blurred DOS
    equals the oracle's (scipy's eigendecomposition of its own tridiagonals); between
    two rounding orders of the same runs the blurred DOS moves by ~1e-15."""
    A = laplacian_2d(30)
    M, n_v = 300, 4
    theta, weight, m_used = ctx.dos_lanczos_ritz(dev(A), M, n_v, seed=2)
    x = np.linspace(-1.0, 9.0, 1001)
    phi = ctx.dos_lanczos_dos(theta, weight, 0.35, x)
    ref = old.lanczos_dos(A, M, n_v, seed=2, sigma=0.35, x=x)
    stats = dict(m_used=m_used.tolist(), w_min=float(weight.min()),
                 sum_err=float(np.abs(weight.sum(axis=1) - 1.0).max()),
                 merged=int(np.sum(weight == 0.0)),
                 theta_desc=float(min(np.diff(theta[l]).min() for l in range(n_v))),
                 dos_rel=float(np.abs(phi - ref).max() / np.abs(ref).max()))
    print("ghost-run figures:", stats)
    # Each weight is the residue of e_1^T (zI - T)^-1 e_1 by a contour integral of the
    # M-step continued fraction, whose FP64 evaluation carries a relative error of
    # about M u (u = 2^-53); so a weight is off by at most ~M u in absolute terms
    # (weights are <= 1) -- nodes whose true weight is ~0 can come out slightly
    # negative -- and the M weights of a run sum to one within ~M^2 u = 1e-11 at
    # M = 300.  Bounds: w >= -M^2 u (-1e-11) and |sum - 1| <= 3 M^2 u (3e-11);
    # measured -2.6e-12 and 8.2e-12.
    ok = (np.all(m_used == M) and stats["w_min"] > -1e-11 and stats["sum_err"] < 3e-11
          and stats["merged"] > 0 and stats["theta_desc"] >= -1e-12 and stats["dos_rel"] < 1e-9)
    assert ok, stats


def test_haydock_matches_continued_fraction(ctx):
    A = anderson_3d(10, 6.0, seed=4)
    theta, weight, _ = ctx.dos_lanczos_ritz(dev(A), 30, 6, seed=3)
    x = np.linspace(-10, 10, 777)
    phi = ctx.dos_haydock_dos(theta, weight, 0.15, x)
    ref = old.haydock_dos(A, 30, 6, seed=3, eta=0.15, x=x)
    assert np.abs(phi - ref).max() < 1e-8 * np.abs(ref).max()


def test_points_error_matches_oracle(ctx):
    A = laplacian_2d(30)
    lam = np.linalg.eigvalsh(A.to_dense())
    lb, ub = -0.08, 8.08
    theta, weight, _ = ctx.dos_lanczos_ritz(dev(A), 40, 10, seed=1)
    e1, einf = ctx.dos_points_error(theta, weight, lb, ub, 0.35, eig=lam)
    x = odos.x_grid(lb, ub, 0.35)
    approx = ctx.dos_lanczos_dos(theta, weight, 0.35, x)
    ref = odos.blurred_exact(lam, 0.35, x)
    diff = np.abs(approx - ref)
    h = x[1] - x[0]
    r1 = h * (diff.sum() - 0.5 * (diff[0] + diff[-1]))
    assert abs(e1 - r1) < 1e-10 and abs(einf - diff.max()) < 1e-10
    # the paper's observation (Section 4): Lanczos is more accurate than KPM at equal M
    mu = ctx.dos_kpm_moments(dev(A), lb, ub, 40, 10, seed=1, precision="f64")
    k1, _ = ctx.dos_smoothed_error(mu, 40, "jackson", lb, ub, 0.35, eig=lam)
    print("M=40, n_v=10, sigma=0.35: E1 Lanczos %.3e vs KPM(Jackson) %.3e" % (e1, k1))
