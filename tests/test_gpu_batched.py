"""Batched sweep (step a8): many matrices of uneven size, one launch per
Chebyshev step for all of them, against the oracle run matrix by matrix with
the same start-vector counters (matrix b uses counter field b)."""
import numpy as np
import pytest

from oracle import bounds as obounds
from oracle import kpm as okpm
from synthetic import anderson_3d, batched_anderson, concat_block_diagonal, laplacian_2d, \
    random_symmetric
from tolerances import fp32_ratio, tol32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1308_5467_gb300 import dos
    c = dos.Context(0)
    yield c
    c.close()


def upload(rp, ci, va, dtype):
    import torch
    from paper_1308_5467_gb300 import dos
    return dos.CSRArrays(int(rp.shape[0] - 1), torch.from_numpy(rp).cuda(),
                         torch.from_numpy(ci).cuda(),
                         torch.from_numpy(va.astype(dtype)).cuda())


def small_batch():
    mats = [anderson_3d(L, W, s) for L, W, s in ((3, 1.0, 1), (7, 16.0, 2), (5, 4.0, 3))]
    mats += [laplacian_2d(9), random_symmetric(40, 0.1, 5, empty_rows=2, long_row=3),
             anderson_3d(9, 8.0, 4), laplacian_2d(1)]
    return mats


def test_bounds_batched_bitwise(ctx):
    mats = small_batch()
    rp, ci, va, seg = concat_block_diagonal(mats)
    for dtype in (np.float64, np.float32):
        lb, ub = ctx.dos_bounds_batched(upload(rp, ci, va, dtype), seg, pad_frac=0.01)
        for b, A in enumerate(mats):
            rlb, rub = obounds.bounds(A.astype(dtype), "gershgorin", pad_frac=0.01)
            if rub > rlb:
                assert (lb[b], ub[b]) == (rlb, rub)
            else:
                assert lb[b] < rlb <= rub < ub[b]


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("M,n_v", [(0, 3), (7, 5), (64, 32), (33, 260)])
def test_small_batch_parity(ctx, precision, M, n_v):
    mats = small_batch()
    rp, ci, va, seg = concat_block_diagonal(mats)
    dtype = np.float64 if precision == "f64" else np.float32
    A = upload(rp, ci, va, dtype)
    lb, ub = ctx.dos_bounds_batched(A, seg, pad_frac=0.02)
    B = len(mats)
    pv = np.empty((B, n_v, M + 1))
    mu = ctx.dos_kpm_moments_batched(A, seg, lb, ub, M, n_v, seed=11, precision=precision,
                                     mu_per_vec=pv)
    for b, Ab in enumerate(mats):
        ref = okpm.kpm_moments_per_vector(Ab.astype(dtype), lb[b], ub[b], M, n_v, seed=11,
                                          batch_index=b)
        tol, tolt = (1e-12, 1e-12) if precision == "f64" else (tol32(M, Ab.n),
                                                               tol32(M, Ab.n * n_v))
        assert np.all(np.abs(pv[b] - ref) <= tol), (b, fp32_ratio(pv[b], ref))
        assert np.all(np.abs(mu[b] - ref.mean(axis=0)) <= tolt), (b, fp32_ratio(mu[b], ref.mean(0)))


def test_batch_of_one_equals_single_call(ctx):
    from paper_1308_5467_gb300 import dos
    A = anderson_3d(8, 3.0, 9)
    Ad = dos.CSRArrays.from_synthetic(A, device="cuda")
    single = ctx.dos_kpm_moments(Ad, -7.6, 7.6, 50, 16, seed=2, precision="f64")
    batched = ctx.dos_kpm_moments_batched(Ad, [0, A.n], [-7.6], [7.6], 50, 16, seed=2,
                                          precision="f64")
    assert np.abs(batched[0] - single).max() < 1e-13


@pytest.fixture(scope="module")
def batch512():
    mats = batched_anderson(512, seed=4)
    return mats, concat_block_diagonal(mats)


def test_full_batch_512_f32_sampled(ctx, batch512):
    """The 512-lattice workload at full size (M = 200, n_v = 32, FP32 SpMM),
    sampled matrices checked against the oracle (all 32 vectors each)."""
    mats, (rp, ci, va, seg) = batch512
    A = upload(rp, ci, va, np.float32)
    lb, ub = ctx.dos_bounds_batched(A, seg, pad_frac=0.01)
    mu = ctx.dos_kpm_moments_batched(A, seg, lb, ub, 200, 32, seed=4, precision="f32")
    assert mu.shape == (512, 201) and np.all(mu[:, 0] == 1.0)
    assert np.all(np.abs(mu) <= 1.0 + 1e-5)
    sizes = np.array([m.n for m in mats])
    picks = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), 0, 255, 511, 100})
    for b in picks:
        ref = okpm.kpm_moments(mats[b].astype(np.float32), lb[b], ub[b], 200, 32, seed=4,
                               batch_index=b, nthreads=8)
        assert np.all(np.abs(mu[b] - ref) <= tol32(200, mats[b].n * 32)), (b, fp32_ratio(mu[b],
                                                                                       ref))


def test_autotuned_shape_gives_same_moments(ctx, batch512):
    mats, (rp, ci, va, seg) = batch512
    A = upload(rp, ci, va, np.float32)
    lb, ub = ctx.dos_bounds_batched(A, seg, pad_frac=0.01)
    default = ctx.dos_kpm_moments_batched(A, seg, lb, ub, 40, 32, seed=4, precision="f32")
    best, ms = ctx.dos_tune(A, 32, "f32", seg_rows=seg)
    assert best["team"] >= 1 and best["tiles"] >= 512 and ms > 0
    tuned = ctx.dos_kpm_moments_batched(A, seg, lb, ub, 40, 32, seed=4, precision="f32")
    # another launch shape groups the FP32 row sums differently: both within the FP32
    # bound of the oracle, so within twice that bound of each other
    n_min = int(np.diff(seg).min())
    assert np.all(np.abs(tuned - default) <= 2 * tol32(40, n_min * 32)), fp32_ratio(tuned, default)
