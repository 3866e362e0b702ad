"""KPML and DGL on the GPU (Sections 3.1.1, 3.1.3, Appendix B) against the oracle.

The library forms the Legendre moments from the doubling Chebyshev sweep and the
exact Legendre-in-Chebyshev expansion; the oracle runs the Legendre vector
recurrence of Algorithm DGL with direct dots.  Agreement at FP64 rounding level
checks both the sweep and the conversion.  KPML, DGL and their error metric
are compared point by point."""
import numpy as np
import pytest
import scipy.special

from oracle import bounds as obounds
from oracle import dos as odos
from oracle import legendre as oleg
from synthetic import anderson_3d, diagonal, laplacian_2d, random_symmetric
from tolerances import fp32_ratio, tol32

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


CASES = {
    "laplacian40": (lambda: laplacian_2d(40), 100, 20, 1),
    "anderson12": (lambda: anderson_3d(12, 6.0, seed=3), 151, 16, 7),
    "random_ragged": (lambda: random_symmetric(777, 0.01, 5, empty_rows=9, long_row=100), 64, 5, 2),
    "one_row": (lambda: diagonal(np.array([0.7])), 6, 3, 4),
}


@pytest.mark.parametrize("name", list(CASES))
def test_legendre_moments_f64_match_oracle(ctx, name):
    make, M, n_v, seed = CASES[name]
    A = make()
    lb, ub = obounds.bounds(A, "gershgorin", pad_frac=0.01)
    if ub <= lb:                               # one eigenvalue: widen by 0.5 per side
        lb, ub = lb - 0.5, ub + 0.5
    pv = np.empty((n_v, M + 1))
    nu = ctx.dos_legendre_moments(dev(A), lb, ub, M, n_v, seed, precision="f64", nu_per_vec=pv)
    ref = oleg.legendre_moments_per_vector(A, lb, ub, M, n_v, seed)
    assert np.abs(pv - ref).max() < 1e-12
    assert np.abs(nu - ref.mean(axis=0)).max() < 1e-12
    assert abs(nu[0] - 1.0) < 1e-14


def test_legendre_moments_f32_form(ctx):
    A = anderson_3d(16, 4.0, seed=2)
    lb, ub = obounds.bounds(A, "gershgorin", pad_frac=0.01)
    M, n_v = 200, 32
    nu = ctx.dos_legendre_moments(dev(A.astype(np.float32)), lb, ub, M, n_v, 2, precision="f32")
    ref = oleg.legendre_moments(A.astype(np.float32), lb, ub, M, n_v, 2)
    # nu_k is a convex combination of mu_0..mu_k (non-negative coefficients summing
    # to one), so its FP32-form error is within the Chebyshev sweep's bound at k
    # (increasing in k), plus the FP64 spread of the two routes
    assert np.all(np.abs(nu - ref) <= tol32(M, A.n * n_v) + 1e-12), fp32_ratio(nu, ref)


def test_conversion_on_exact_moments(ctx):
    vals = np.linspace(-0.99, 0.97, 301) ** 3
    M = 400
    th = np.arccos(vals)
    mu = np.array([np.mean(np.cos(k * th)) for k in range(M + 1)])
    nu = ctx.dos_cheb_to_legendre(mu)
    ref = np.array([np.mean(scipy.special.eval_legendre(k, vals)) for k in range(M + 1)])
    assert np.abs(nu - ref).max() < 1e-13
    # several rows at once, device in and out
    import torch
    rows = torch.tensor(np.stack([mu, mu[::-1].copy(), np.zeros(M + 1)]), device="cuda")
    out = ctx.dos_cheb_to_legendre(rows).cpu().numpy()
    assert np.abs(out[0] - ref).max() < 1e-13
    assert np.all(out[2] == 0.0)


def test_kpml_reconstruct_matches_oracle(ctx):
    A = anderson_3d(10, 5.0, seed=1)
    lb, ub = obounds.bounds(A, "gershgorin", pad_frac=0.01)
    M = 80
    nu = oleg.legendre_moments(A, lb, ub, M, 8, 3)
    t = np.linspace(-1.0, 1.0, 513)
    phi, phil = ctx.dos_kpml_reconstruct(nu, lb, ub, t=t, want_lambda=True)
    ref = oleg.kpml(nu, t)
    assert np.abs(phi - ref).max() < 1e-12 * np.abs(ref).max()
    assert np.abs(phil - ref / (0.5 * (ub - lb))).max() < 1e-12 * np.abs(ref).max()
    # default grid: Chebyshev nodes
    phi_n = ctx.dos_kpml_reconstruct(nu, N_t=300)
    assert np.abs(phi_n - oleg.kpml(nu, odos.chebyshev_nodes(300))).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("sigma,tol", [(0.35, 1e-6), (0.1, 1e-6), (0.35, 1e-8)])
def test_dgl_matches_oracle(ctx, sigma, tol):
    A = laplacian_2d(24)
    lb, ub = -0.08, 8.08
    M = 300
    nu = oleg.legendre_moments(A, lb, ub, M, 10, 1)
    x = np.linspace(lb - 1.0, ub + 1.0, 1501)
    phi, used = ctx.dos_dgl(nu, lb, ub, sigma, tol=tol, x=x)
    ref, ref_used = oleg.dgl_lambda(nu, lb, ub, sigma, x, tol=tol)
    same = used == ref_used
    # the stop test can flip at a rounding-level tie; the rest must agree closely
    assert same.mean() > 0.99
    scale = np.abs(ref).max()
    # Eq. Leg3 amplifies rounding as k grows (Appendix B): up to the paper's stop
    # (tol 1e-6) gamma_k keeps ~1e-12 absolute accuracy, with tol 1e-8 the recurrence
    # runs ~10 steps further and its own error reaches ~1e-9 (oracle vs quadrature of
    # Eq. DGLcoeff), so the two sides' rounding (erf/exp and operation order) can differ
    # by that much times (k + 1/2) / (sqrt(2 pi) sigma).
    rel = 1e-10 if tol >= 1e-6 else 1e-7
    assert np.abs(phi[same] - ref[same]).max() < rel * scale
    slack = (ref_used.max() + 2) * tol / (np.sqrt(2 * np.pi) * sigma) * 2
    assert np.abs(phi - ref).max() < rel * scale + slack
    # the metric-grid default
    phi_g, _ = ctx.dos_dgl(nu, lb, ub, sigma, tol=tol, N_x=4000)
    ref_g, _ = oleg.dgl_lambda(nu, lb, ub, sigma, odos.x_grid(lb, ub, sigma), tol=tol)
    assert np.abs(phi_g - ref_g).max() < rel * scale + slack


@pytest.mark.parametrize("method", ["kpml", "dgl"])
def test_legendre_error_matches_oracle(ctx, method):
    A = laplacian_2d(20)
    lam = np.linalg.eigvalsh(A.to_dense())
    lb, ub = -0.08, 8.08
    M = 60
    nu = oleg.legendre_moments(A, lb, ub, M, 12, 5)
    e1, einf = ctx.dos_legendre_error(nu, method, lb, ub, 0.35, eig=lam)
    r1, rinf = oleg.legendre_error(nu, method, lb, ub, 0.35, eigs=lam)
    assert abs(e1 - r1) < 1e-9 * max(r1, 1e-3) + 1e-12
    assert abs(einf - rinf) < 1e-9 * max(rinf, 1e-3) + 1e-12
    # against reference Chebyshev moments
    from oracle import kpm as okpm
    ref_mu = okpm.kpm_moments(A, lb, ub, 120, 12, 5)
    e1, _ = ctx.dos_legendre_error(nu, method, lb, ub, 0.35, ref_mu=ref_mu)
    r1, _ = oleg.legendre_error(nu, method, lb, ub, 0.35, ref_mu=ref_mu)
    assert abs(e1 - r1) < 1e-9 * max(r1, 1e-3) + 1e-12


def test_laplacian_methods_side_by_side(ctx):
    """Section 4.1's comparison on the 40x40 Laplacian, M = 100, n_v = 20: KPM
    without damping, KPML and DGL behave alike; printed for the record."""
    A = laplacian_2d(40)
    lam = np.linalg.eigvalsh(A.to_dense())
    lb, ub = -0.08, 8.08
    Ad = dev(A)
    mu = ctx.dos_kpm_moments(Ad, lb, ub, 100, 20, 1, precision="f64")
    nu = ctx.dos_legendre_moments(Ad, lb, ub, 100, 20, 1, precision="f64")
    out = {}
    for sigma in (0.35, 0.05):
        out[("kpm", sigma)] = ctx.dos_smoothed_error(mu, 100, "none", lb, ub, sigma, eig=lam)[1]
        out[("kpml", sigma)] = ctx.dos_legendre_error(nu, "kpml", lb, ub, sigma, eig=lam)[1]
        out[("dgl", sigma)] = ctx.dos_legendre_error(nu, "dgl", lb, ub, sigma, eig=lam)[1]
    print("E_inf at M=100, n_v=20:", {f"{k[0]}@{k[1]}": round(v, 5) for k, v in out.items()})
    for sigma in (0.35, 0.05):
        vals = [out[(m, sigma)] for m in ("kpm", "kpml", "dgl")]
        assert max(vals) < 3 * min(vals)


def test_bad_inputs(ctx):
    from paper_1308_5467_gb300 import dos
    nu = np.ones(5)
    with pytest.raises(dos.DosError):
        ctx.dos_legendre_error(nu, 7, -1.0, 1.0, 0.1, eig=np.zeros(3))
    with pytest.raises(dos.DosError):
        ctx.dos_dgl(nu, 1.0, -1.0, 0.1)
    with pytest.raises(dos.DosError):
        ctx.dos_dgl(nu, -1.0, 1.0, 0.0)
    with pytest.raises(dos.DosError):
        ctx.dos_kpml_reconstruct(nu, 1.0, 1.0, N_t=10, want_lambda=True)
