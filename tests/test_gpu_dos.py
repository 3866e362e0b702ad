"""Parity of bounds (step a1), reconstruction (a6) and the smoothed error (a7)
with the CPU oracle, through the C ABI."""
import numpy as np
import pytest

from oracle import bounds as obounds
from oracle import dos as odos
from oracle import kpm as okpm
from synthetic import anderson_3d, chung_lu_normalized_laplacian, diagonal, laplacian_2d, \
    random_symmetric

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1308_5467_gb300 import dos
    c = dos.Context(0)
    yield c
    c.close()


def dev(A, dtype=None):
    from paper_1308_5467_gb300 import dos
    return dos.CSRArrays.from_synthetic(A, device="cuda", dtype=dtype)


@pytest.mark.parametrize("make", [lambda: laplacian_2d(40), lambda: anderson_3d(12, 4.0, 1),
                                  lambda: random_symmetric(200, 0.03, 4, empty_rows=5, long_row=9),
                                  lambda: chung_lu_normalized_laplacian(3000, seed=5),
                                  lambda: diagonal(np.array([2.5]))])
def test_gershgorin_bitwise(ctx, make):
    A = make()
    for dtype in (np.float64, np.float32):
        Aw = A.astype(dtype)
        got = ctx.dos_bounds(dev(Aw), "gershgorin", pad_frac=0.01)
        ref = obounds.bounds(Aw, "gershgorin", pad_frac=0.01)
        if ref[1] > ref[0]:
            assert got == ref
        else:  # single eigenvalue: widened to a unit interval around it
            assert got[0] < ref[0] <= ref[1] < got[1]


@pytest.mark.parametrize("steps", [1, 5, 20, 64])
@pytest.mark.parametrize("make", [lambda: laplacian_2d(40), lambda: anderson_3d(10, 6.0, 2),
                                  lambda: random_symmetric(150, 0.05, 9, empty_rows=3)])
def test_lanczos_bounds_match_oracle(ctx, make, steps):
    A = make()
    got = ctx.dos_bounds(dev(A), "lanczos", steps=steps, seed=3, pad_frac=0.0)
    ref = obounds.bounds(A, "lanczos", steps=steps, seed=3, pad_frac=0.0)
    scale = max(abs(ref[0]), abs(ref[1]), 1.0)
    assert abs(got[0] - ref[0]) < 1e-9 * scale and abs(got[1] - ref[1]) < 1e-9 * scale


def test_lanczos_encloses_spectrum_when_padded(ctx):
    A = anderson_3d(12, 4.0, 6)
    lam = np.linalg.eigvalsh(A.to_dense())
    lb, ub = ctx.dos_bounds(dev(A), "lanczos", steps=30, seed=1, pad_frac=0.01)
    assert lb <= lam[0] and ub >= lam[-1]


def test_lanczos_invariant_subspace_stops_early(ctx):
    # A diagonal matrix with 3 distinct values: the Krylov space has dimension 3.
    A = diagonal(np.repeat([1.0, 2.0, 4.0], 50))
    lb, ub = ctx.dos_bounds(dev(A), "lanczos", steps=20, seed=0, pad_frac=0.0)
    assert abs(lb - 1.0) < 1e-9 and abs(ub - 4.0) < 1e-9


@pytest.mark.parametrize("damping", ["jackson", "none"])
@pytest.mark.parametrize("M,N_t", [(0, 10), (1, 7), (100, 1000), (256, 256), (1000, 333)])
def test_reconstruct_parity(ctx, damping, M, N_t):
    rng = np.random.default_rng(M + N_t)
    mu = np.concatenate([[1.0], rng.uniform(-0.3, 0.3, M) / (1 + np.arange(M))])
    phi, phil = ctx.dos_reconstruct(mu, M, damping, -2.0, 6.0, N_t=N_t, want_lambda=True)
    _, rphi, rphil = odos.reconstruct(mu, damping, N_t=N_t, lb=-2.0, ub=6.0)
    scale = np.abs(rphi).max()
    assert np.abs(phi - rphi).max() < 1e-11 * scale
    assert np.abs(phil - rphil).max() < 1e-11 * scale / 4.0
    t = np.linspace(-0.999, 0.999, 77)
    phi_t = ctx.dos_reconstruct(mu, M, damping, t=t)
    _, rt, _ = odos.reconstruct(mu, damping, t=t)
    assert np.abs(phi_t - rt).max() < 1e-11 * np.abs(rt).max()


def test_smoothed_error_parity_vs_eigenvalues(ctx):
    A = laplacian_2d(40)
    lam = np.linalg.eigvalsh(A.to_dense())
    lb, ub = -0.08, 8.08
    mu = okpm.kpm_moments(A, lb, ub, 100, 20, seed=1)
    for sigma in (0.35, 0.05):
        for damping in ("jackson", "none"):
            got = ctx.dos_smoothed_error(mu, 100, damping, lb, ub, sigma, eig=lam)
            ref = odos.smoothed_error(mu, damping, lb, ub, sigma, eigs=lam)
            assert abs(got[0] - ref[0]) < 1e-10 and abs(got[1] - ref[1]) < 1e-9


def test_smoothed_error_parity_vs_reference_moments(ctx):
    A = anderson_3d(14, 4.0, 3)
    lb, ub = obounds.bounds(A, "gershgorin", pad_frac=0.01)
    mu = okpm.kpm_moments(A, lb, ub, 150, 4, seed=1)
    ref_mu = okpm.kpm_moments(A, lb, ub, 300, 64, seed=99)
    sigma = 0.02 * (ub - lb)
    got = ctx.dos_smoothed_error(mu, 150, "jackson", lb, ub, sigma, ref_mu=ref_mu)
    ref = odos.smoothed_error(mu, "jackson", lb, ub, sigma, ref_mu=ref_mu)
    assert abs(got[0] - ref[0]) < 1e-10 and abs(got[1] - ref[1]) < 1e-9
    same = ctx.dos_smoothed_error(ref_mu, 300, "jackson", lb, ub, sigma, ref_mu=ref_mu)
    assert same == (0.0, 0.0)


def test_reconstruct_device_tensors(ctx):
    import torch
    mu = torch.tensor(np.r_[1.0, 0.2, -0.1, 0.05], dtype=torch.float64, device="cuda")
    out = torch.empty(64, dtype=torch.float64, device="cuda")
    ctx.dos_reconstruct(mu, 3, "jackson", phi_hat=out, N_t=64)
    _, ref, _ = odos.reconstruct(mu.cpu().numpy(), "jackson", N_t=64)
    assert np.abs(out.cpu().numpy() - ref).max() < 1e-12


@pytest.mark.parametrize("damping", ["jackson", "none"])
def test_reconstruct_batched_rows_equal_single_calls(ctx, damping):
    """dos_reconstruct_batched: every row bit for bit as dos_reconstruct of that row
    (same kernels' arithmetic), host and device arrays, default and given grids;
    and within 1e-12 of the oracle's reconstruction."""
    import torch
    rng = np.random.default_rng(3)
    B, M = 37, 120
    mu = np.concatenate([np.ones((B, 1)), rng.uniform(-0.3, 0.3, (B, M))], axis=1)
    t = np.sort(rng.uniform(-0.99, 0.99, 77))
    for grid in (None, t):
        out = ctx.dos_reconstruct_batched(mu, damping, t=grid, N_t=256)
        for b in (0, 17, B - 1):
            single = ctx.dos_reconstruct(mu[b], M, damping, t=grid, N_t=256)
            assert np.array_equal(out[b], single)
            _, ref, _ = odos.reconstruct(mu[b], damping, t=grid, N_t=256)
            assert np.abs(out[b] - ref).max() < 1e-12 * np.abs(ref).max()
    dmu = torch.from_numpy(mu).cuda()
    dout = torch.empty((B, 256), dtype=torch.float64, device="cuda")
    ctx.dos_reconstruct_batched(dmu, damping, N_t=256, phi_hat=dout)
    torch.cuda.synchronize()
    assert np.array_equal(dout.cpu().numpy(), ctx.dos_reconstruct_batched(mu, damping, N_t=256))
