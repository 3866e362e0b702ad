"""Parity of the CUDA moment sweep (steps a2-a5) with the CPU oracle.

Every comparison runs the library through its C ABI (ctypes binding) and the
oracle on the same seeded inputs.  Tolerances (tests/tolerances.py, with the
error model): FP64 form 1e-12 absolute per moment; FP32 form
u sqrt(k+1) (1/2 + 40/sqrt(N)), u = 2^-24, N the (row, vector) terms a moment
averages, against the FP64 oracle run on the FP32-rounded matrix values.
"""
import numpy as np
import pytest

from oracle import bounds as obounds
from oracle import kpm as okpm
from synthetic import anderson_3d, laplacian_2d, random_symmetric, diagonal
from tolerances import TOL64, fp32_ratio, tol32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1308_5467_gb300 import dos
    c = dos.Context(0)
    yield c
    c.close()


def dev(A, dtype=None):
    from paper_1308_5467_gb300 import dos
    return dos.CSRArrays.from_synthetic(A, device="cuda", dtype=dtype)


def test_start_vectors_golden(ctx):
    rows = np.loadtxt("tests/golden/rademacher_signs.txt", dtype=np.int64)
    for seed in np.unique(rows[:, 0]):
        for b in np.unique(rows[:, 1]):
            sel = rows[(rows[:, 0] == seed) & (rows[:, 1] == b)]
            V = ctx.dos_start_vectors(16, 256, int(seed), batch_index=int(b))
            for _, _, l, i, v in sel:
                assert V[i, l] == v


@pytest.mark.parametrize("n_v,off", [(1, 0), (5, 3), (64, 0), (100, 61), (300, 0)])
def test_start_vectors_match_oracle(ctx, n_v, off):
    V = ctx.dos_start_vectors(777, n_v, 42, batch_index=2, vec_offset=off)
    W = okpm.start_block(777, n_v, 42, batch_index=2, vec_offset=off)
    assert np.array_equal(V, W)
    V32 = ctx.dos_start_vectors(777, n_v, 42, batch_index=2, vec_offset=off, dtype="float32")
    assert np.array_equal(V32.astype(np.float64), W)


def test_laplacian_40x40_f64_full_config(ctx):
    """Config 1 at its full size: n = 1600, M = 100, n_v = 20, FP64."""
    A = laplacian_2d(40)
    lb, ub = -0.08, 8.08
    pv = np.empty((20, 101))
    mu = ctx.dos_kpm_moments(dev(A), lb, ub, 100, 20, seed=1, precision="f64", mu_per_vec=pv)
    ref = okpm.kpm_moments_per_vector(A, lb, ub, 100, 20, seed=1)
    assert np.abs(pv - ref).max() < TOL64
    assert np.abs(mu - ref.mean(axis=0)).max() < TOL64
    assert mu[0] == 1.0


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_matrix_without_nonzeros(ctx, precision):
    """nnz = 0: every eigenvalue is 0, so for any start vectors mu_k = T_k(-c/d)
    exactly; with bounds [-1, 1], T_k(0) = cos(k pi / 2)."""
    from synthetic.matrices import CSR
    n = 50
    A = CSR(n, np.zeros(n + 1, dtype=np.int32), np.zeros(0, dtype=np.int32),
            np.zeros(0, dtype=np.float64), {"family": "zero"})
    dtype = np.float64 if precision == "f64" else np.float32
    mu = ctx.dos_kpm_moments(dev(A, dtype), -1.0, 1.0, 9, 5, seed=3, precision=precision)
    assert np.array_equal(mu, np.round(np.cos(np.arange(10) * np.pi / 2)))
    ref = okpm.kpm_moments(A, -1.0, 1.0, 9, 5, seed=3)
    assert np.array_equal(ref, mu)
    lb, ub = ctx.dos_bounds(dev(A, dtype), "gershgorin", pad_frac=0.01)
    assert (lb, ub) == (-0.5, 0.5)           # a single eigenvalue gets +-0.5


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("n,M,n_v", [(1, 5, 3), (37, 0, 4), (37, 1, 4), (37, 2, 7), (97, 33, 1),
                                     (97, 64, 20), (300, 81, 33), (513, 50, 64)])
def test_random_ragged_parity(ctx, precision, n, M, n_v):
    """Tiny to multi-tile sizes, empty rows, one dense row, odd/even M, ragged n_v."""
    if n == 1:
        A = diagonal(np.array([0.7]))
    else:
        A = random_symmetric(n, min(0.2, 6.0 / n), seed=n + M, empty_rows=max(1, n // 20),
                             long_row=n // 3)
    lam = np.linalg.eigvalsh(A.to_dense())
    lb, ub = lam[0] - 0.05 * (lam[-1] - lam[0] + 1), lam[-1] + 0.05 * (lam[-1] - lam[0] + 1)
    vals = np.float64 if precision == "f64" else np.float32
    Aw = A.astype(vals)
    pv = np.empty((n_v, M + 1))
    mu = ctx.dos_kpm_moments(dev(Aw), lb, ub, M, n_v, seed=7, precision=precision, mu_per_vec=pv)
    ref = okpm.kpm_moments_per_vector(Aw, lb, ub, M, n_v, seed=7)
    tol, tolt = (TOL64, TOL64) if precision == "f64" else (tol32(M, n), tol32(M, n * n_v))
    assert np.all(np.abs(pv - ref) <= tol), fp32_ratio(pv, ref)
    assert np.all(np.abs(mu - ref.mean(axis=0)) <= tolt), fp32_ratio(mu, ref.mean(axis=0))


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_host_and_device_inputs_agree_and_deterministic(ctx, precision):
    from paper_1308_5467_gb300 import dos
    A = anderson_3d(9, 4.0, seed=5)
    lb, ub = -8.2, 8.2
    Ad = dev(A)
    Ah = dos.CSRArrays.from_synthetic(A)  # host arrays, copied by the library
    a = ctx.dos_kpm_moments(Ad, lb, ub, 77, 12, seed=3, precision=precision)
    b = ctx.dos_kpm_moments(Ah, lb, ub, 77, 12, seed=3, precision=precision)
    c = ctx.dos_kpm_moments(Ad, lb, ub, 77, 12, seed=3, precision=precision)
    assert np.array_equal(a, b) and np.array_equal(a, c)


def test_device_output_tensor(ctx):
    import torch
    A = laplacian_2d(12)
    out = torch.empty(41, dtype=torch.float64, device="cuda")
    ctx.dos_kpm_moments(dev(A), -0.1, 8.1, 40, 6, seed=2, precision="f64", mu=out)
    ref = okpm.kpm_moments(A, -0.1, 8.1, 40, 6, seed=2)
    assert np.abs(out.cpu().numpy() - ref).max() < TOL64


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_vector_panels_large_n_v(ctx, precision):
    """n_v above one panel (256 vectors): panels of the block are swept in turn."""
    A = anderson_3d(6, 3.0, seed=1)
    lb, ub = -7.8, 7.8
    n_v, M = 700, 20
    pv = np.empty((n_v, M + 1))
    mu = ctx.dos_kpm_moments(dev(A), lb, ub, M, n_v, seed=4, precision=precision, mu_per_vec=pv)
    ref = okpm.kpm_moments_per_vector(A.astype(np.float32) if precision == "f32" else A,
                                      lb, ub, M, n_v, seed=4)
    tol, tolt = (TOL64, TOL64) if precision == "f64" else (tol32(M, A.n), tol32(M, A.n * n_v))
    assert np.all(np.abs(pv - ref) <= tol), fp32_ratio(pv, ref)
    assert np.all(np.abs(mu - ref.mean(axis=0)) <= tolt), fp32_ratio(mu, ref.mean(axis=0))


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("n_v,launch", [
    (64, {"panel": 4}), (64, {"panel": 8}), (64, {"panel": 16}),
    (64, {"panel": 16, "staged": 3}), (64, {"panel": 16, "staged": 4}),
    (64, {"panel": 16, "chunk_bytes": 32}), (64, {"panel": 32, "tiles": 5}),
    (20, {"panel": 4}), (20, {"panel": 8}), (20, {"panel": 16})])
def test_narrow_vector_panels_parity(ctx, precision, n_v, launch):
    """Vectors swept in narrower panels (launch.panel: ceil(n_v / w) passes over A
    of equal width, the last possibly narrower; 20 vectors in panels of 8 are three
    of 7): per-vector and total moments against the oracle, on a lattice and on a
    random matrix with empty rows and a dense row; the totals agree with the
    one-pass sweep up to the order of their FP64 sums."""
    dtype = np.float64 if precision == "f64" else np.float32
    for A, lb, ub in ((anderson_3d(11, 6.0, seed=4), -9.6, 9.6),
                      (random_symmetric(300, 0.03, 5, empty_rows=5, long_row=41), None, None)):
        Aw = A.astype(dtype)
        if lb is None:
            lb, ub = obounds.bounds(A, "gershgorin", pad_frac=0.01)
        M = 41
        pv = np.empty((n_v, M + 1))
        mu = ctx.dos_kpm_moments(dev(Aw), lb, ub, M, n_v, seed=6, precision=precision,
                                 launch=launch, mu_per_vec=pv)
        mu_tot = ctx.dos_kpm_moments(dev(Aw), lb, ub, M, n_v, seed=6, precision=precision,
                                     launch=launch)
        one_pass = ctx.dos_kpm_moments(dev(Aw), lb, ub, M, n_v, seed=6, precision=precision)
        ref = okpm.kpm_moments_per_vector(Aw, lb, ub, M, n_v, seed=6)
        tol, tolt = (TOL64, TOL64) if precision == "f64" else (tol32(M, A.n),
                                                               tol32(M, A.n * n_v))
        assert np.all(np.abs(pv - ref) <= tol), fp32_ratio(pv, ref)
        assert np.all(np.abs(mu - ref.mean(axis=0)) <= tolt), fp32_ratio(mu, ref.mean(0))
        assert np.all(np.abs(mu_tot - ref.mean(axis=0)) <= tolt), fp32_ratio(mu_tot, ref.mean(0))
        if precision == "f64":
            assert np.abs(mu_tot - one_pass).max() < 1e-13


def test_tuned_shape_with_narrower_panels(ctx):
    """The autotuner's shape (one pass: panel 0) and the same shape with the vectors
    split into panels of 16 both match the oracle."""
    A = anderson_3d(12, 5.0, seed=2).astype(np.float32)
    shape, ms = ctx.dos_tune(dev(A), 48, "f32")
    assert shape["panel"] == 0 and ms > 0
    ref = okpm.kpm_moments(A, -9.0, 9.0, 30, 48, seed=2)
    for launch in (shape, {**{k: v for k, v in shape.items() if k != "tiles"}, "panel": 16}):
        mu = ctx.dos_kpm_moments(dev(A), -9.0, 9.0, 30, 48, seed=2, precision="f32",
                                 launch=launch)
        assert np.all(np.abs(mu - ref) <= tol32(30, A.n * 48)), fp32_ratio(mu, ref)


def test_vec_offset_shards_union(ctx):
    A = laplacian_2d(15)
    full = np.empty((10, 31))
    ctx.dos_kpm_moments(dev(A), -0.1, 8.1, 30, 10, seed=9, precision="f64", mu_per_vec=full)
    part = np.empty((4, 31))
    ctx.dos_kpm_moments(dev(A), -0.1, 8.1, 30, 4, seed=9, precision="f64", mu_per_vec=part,
                        vec_offset=6)
    assert np.abs(full[6:] - part).max() < 1e-13


@pytest.mark.parametrize("launch", [{"team": 16, "chunks": 4}, {"team": 32, "chunks": 1},
                                    {"team": 16, "chunks": 2, "tiles": 7},
                                    {"team": 8, "chunks": 4, "tiles": 1000}])
def test_launch_shapes_agree(ctx, launch):
    A = anderson_3d(10, 6.0, seed=3)
    lb, ub = -9.5, 9.5
    ref = okpm.kpm_moments(A, lb, ub, 60, 64, seed=5)
    mu = ctx.dos_kpm_moments(dev(A), lb, ub, 60, 64, seed=5, precision="f64", launch=launch)
    assert np.abs(mu - ref).max() < TOL64


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("launch", [{"staged": 2}, {"team": 8, "chunks": 2, "staged": 2},
                                    {"team": 32, "chunks": 1, "staged": 2, "tiles": 5},
                                    {"team": 16, "chunks": 1, "staged": 2, "tiles": 333}])
def test_staged_panels_parity(ctx, precision, launch):
    """Row panels staged in shared memory by bulk asynchronous copies (staged 2):
    ragged last panels and chunks, one tile of many rows, many small tiles,
    ragged n_v."""
    A = anderson_3d(13, 6.0, seed=4)
    lb, ub = -9.6, 9.6
    dtype = np.float64 if precision == "f64" else np.float32
    Aw = A.astype(dtype)
    for n_v in (64, 20):
        if launch.get("team", 16) * launch.get("chunks", 1) * (2 if precision == "f64" else 4) < n_v:
            continue
        pv = np.empty((n_v, 71))
        mu = ctx.dos_kpm_moments(dev(Aw), lb, ub, 70, n_v, seed=5, precision=precision,
                                 launch=launch, mu_per_vec=pv)
        mu_tot = ctx.dos_kpm_moments(dev(Aw), lb, ub, 70, n_v, seed=5, precision=precision,
                                     launch=launch)
        ref = okpm.kpm_moments_per_vector(Aw, lb, ub, 70, n_v, seed=5)
        tol, tolt = (TOL64, TOL64) if precision == "f64" else (tol32(70, A.n),
                                                               tol32(70, A.n * n_v))
        assert np.all(np.abs(pv - ref) <= tol), fp32_ratio(pv, ref)
        assert np.all(np.abs(mu - ref.mean(axis=0)) <= tolt)
        assert np.all(np.abs(mu_tot - ref.mean(axis=0)) <= tolt), fp32_ratio(mu_tot, ref.mean(0))


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("launch", [{"chunk_bytes": 32},
                                    {"team": 4, "chunks": 2, "chunk_bytes": 32},
                                    {"team": 8, "chunks": 1, "chunk_bytes": 32, "tiles": 7},
                                    {"team": 16, "chunks": 2, "chunk_bytes": 32, "tiles": 500},
                                    {"team": 2, "chunks": 2, "chunk_bytes": 32}])
def test_wide_chunk_parity(ctx, precision, launch):
    """32-byte chunks (256-bit loads and stores): per-vector and total moments,
    several tile counts, n_v whose padded row is whole 32-byte chunks (64, 24 in
    FP32; 64, 20 in FP64); shapes that do not cover the row are rejected."""
    from paper_1308_5467_gb300 import dos
    A = anderson_3d(13, 6.0, seed=4)
    lb, ub = -9.6, 9.6
    dtype = np.float64 if precision == "f64" else np.float32
    Aw = A.astype(dtype)
    per_chunk = 4 if precision == "f64" else 8
    for n_v in ((64, 20) if precision == "f64" else (64, 24)):
        if launch.get("team", 0) * launch.get("chunks", 1) * per_chunk < n_v and "team" in launch:
            with pytest.raises(dos.DosError):
                ctx.dos_kpm_moments(dev(Aw), lb, ub, 70, n_v, seed=5, precision=precision,
                                    launch=launch)
            continue
        pv = np.empty((n_v, 71))
        mu = ctx.dos_kpm_moments(dev(Aw), lb, ub, 70, n_v, seed=5, precision=precision,
                                 launch=launch, mu_per_vec=pv)
        mu_tot = ctx.dos_kpm_moments(dev(Aw), lb, ub, 70, n_v, seed=5, precision=precision,
                                     launch=launch)
        ref = okpm.kpm_moments_per_vector(Aw, lb, ub, 70, n_v, seed=5)
        tol, tolt = (TOL64, TOL64) if precision == "f64" else (tol32(70, A.n),
                                                               tol32(70, A.n * n_v))
        assert np.all(np.abs(pv - ref) <= tol), fp32_ratio(pv, ref)
        assert np.all(np.abs(mu - ref.mean(axis=0)) <= tolt)
        assert np.all(np.abs(mu_tot - ref.mean(axis=0)) <= tolt), fp32_ratio(mu_tot, ref.mean(0))


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("launch", [{"staged": 3}, {"team": 16, "chunks": 1, "staged": 3},
                                    {"team": 8, "chunks": 2, "staged": 3, "tiles": 7},
                                    {"team": 32, "chunks": 2, "staged": 3, "tiles": 500},
                                    {"team": 32, "chunks": 4, "staged": 3},
                                    {"team": 16, "chunks": 1, "staged": 3, "depth": 8},
                                    {"team": 16, "chunks": 2, "staged": 3, "depth": 2,
                                     "tiles": 3}])
def test_tma_gather_parity(ctx, precision, launch):
    """Rows gathered by TMA (tile::gather4, four nonzeros per copy, a ring of 2, 4 or
    8 batches per team running ahead across rows): a lattice, and a random matrix with
    empty rows and one dense row (batches padded past the row's end), per-vector and
    total moments, several tile counts and n_v."""
    from paper_1308_5467_gb300 import dos
    dtype = np.float64 if precision == "f64" else np.float32
    per_chunk = 2 if precision == "f64" else 4
    for A, lb, ub in ((anderson_3d(13, 6.0, seed=4), -9.6, 9.6),
                      (random_symmetric(400, 0.02, 9, empty_rows=7, long_row=37), None, None)):
        Aw = A.astype(dtype)
        if lb is None:
            lb, ub = obounds.bounds(A, "gershgorin", pad_frac=0.01)
        for n_v in (64, 20):
            if "team" in launch and launch["team"] * launch.get("chunks", 1) * per_chunk < n_v:
                with pytest.raises(dos.DosError):
                    ctx.dos_kpm_moments(dev(Aw), lb, ub, 30, n_v, seed=5, precision=precision,
                                        launch=launch)
                continue
            pv = np.empty((n_v, 71))
            mu = ctx.dos_kpm_moments(dev(Aw), lb, ub, 70, n_v, seed=5, precision=precision,
                                     launch=launch, mu_per_vec=pv)
            mu_tot = ctx.dos_kpm_moments(dev(Aw), lb, ub, 70, n_v, seed=5, precision=precision,
                                         launch=launch)
            ref = okpm.kpm_moments_per_vector(Aw, lb, ub, 70, n_v, seed=5)
            tol, tolt = (TOL64, TOL64) if precision == "f64" else (tol32(70, A.n),
                                                                   tol32(70, A.n * n_v))
            assert np.all(np.abs(pv - ref) <= tol), fp32_ratio(pv, ref)
            assert np.all(np.abs(mu - ref.mean(axis=0)) <= tolt)
            assert np.all(np.abs(mu_tot - ref.mean(axis=0)) <= tolt), fp32_ratio(mu_tot,
                                                                                 ref.mean(0))


def test_tma_gather_wait_timeout_is_reported(ctx):
    """The TMA-gather kernel's bounded wait made to run out (the barrier is armed
    and no gather issued): DOS_ETIMEOUT, and the context still works."""
    from paper_1308_5467_gb300 import dos
    A = dev(anderson_3d(8, 6.0, seed=4))
    with pytest.raises(dos.DosError) as ei:
        ctx.dos_kpm_moments(A, -9.6, 9.6, 10, 16, seed=5, precision="f64",
                            launch={"staged": 3}, flags=dos.DOS_OPT_TEST_STALL_WAIT,
                            wait_limit_cycles=2_000_000)
    assert ei.value.status == dos.DOS_ETIMEOUT
    mu = ctx.dos_kpm_moments(A, -9.6, 9.6, 10, 16, seed=5, precision="f64", launch={"staged": 3})
    ref = okpm.kpm_moments(anderson_3d(8, 6.0, seed=4), -9.6, 9.6, 10, 16, seed=5)
    assert np.abs(mu - ref).max() < TOL64


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("launch", [{"staged": 4}, {"team": 8, "chunks": 2, "staged": 4},
                                    {"team": 4, "chunks": 2, "chunk_bytes": 32, "staged": 4},
                                    {"team": 16, "chunks": 1, "staged": 4, "tiles": 2},
                                    {"team": 8, "chunks": 2, "staged": 4, "tiles": 500},
                                    {"team": 32, "chunks": 1, "chunk_bytes": 32, "staged": 4}])
def test_csr_staged_parity(ctx, precision, launch):
    """Each tile's CSR slice staged in shared memory by bulk copies (staged 4): a
    lattice, a random matrix with empty rows and one dense row (nnz not a multiple of
    four: the slice's tail comes from plain loads), tiles too large to stage (two
    tiles: they read the CSR from global memory), many small tiles; per-vector and
    total moments."""
    from paper_1308_5467_gb300 import dos
    dtype = np.float64 if precision == "f64" else np.float32
    per_chunk = launch.get("chunk_bytes", 16) // (8 if precision == "f64" else 4)
    mats = ((anderson_3d(13, 6.0, seed=4), -9.6, 9.6),
            (random_symmetric(401, 0.02, 9, empty_rows=7, long_row=37), None, None),
            (diagonal(np.linspace(-1.0, 1.0, 5003)), -1.1, 1.1))
    for A, lb, ub in mats:
        Aw = A.astype(dtype)
        if lb is None:
            lb, ub = obounds.bounds(A, "gershgorin", pad_frac=0.01)
        for n_v in (64, 24):
            ok_shape = ("team" not in launch or
                        launch["team"] * launch.get("chunks", 1) * per_chunk >= n_v) and \
                (n_v * (8 if precision == "f64" else 4)) % launch.get("chunk_bytes", 16) == 0
            if not ok_shape:
                with pytest.raises(dos.DosError):
                    ctx.dos_kpm_moments(dev(Aw), lb, ub, 30, n_v, seed=5, precision=precision,
                                        launch=launch)
                continue
            pv = np.empty((n_v, 71))
            mu = ctx.dos_kpm_moments(dev(Aw), lb, ub, 70, n_v, seed=5, precision=precision,
                                     launch=launch, mu_per_vec=pv)
            mu_tot = ctx.dos_kpm_moments(dev(Aw), lb, ub, 70, n_v, seed=5, precision=precision,
                                         launch=launch)
            ref = okpm.kpm_moments_per_vector(Aw, lb, ub, 70, n_v, seed=5)
            tol, tolt = (TOL64, TOL64) if precision == "f64" else (tol32(70, A.n),
                                                                   tol32(70, A.n * n_v))
            assert np.all(np.abs(pv - ref) <= tol), fp32_ratio(pv, ref)
            assert np.all(np.abs(mu - ref.mean(axis=0)) <= tolt)
            assert np.all(np.abs(mu_tot - ref.mean(axis=0)) <= tolt), fp32_ratio(mu_tot,
                                                                                 ref.mean(0))


def test_csr_staged_wait_timeout_is_reported(ctx):
    """The CSR-staged kernel's bounded wait made to run out (it expects 16 bytes more
    than it copies): DOS_ETIMEOUT, and the context still works."""
    from paper_1308_5467_gb300 import dos
    A = dev(anderson_3d(8, 6.0, seed=4))
    with pytest.raises(dos.DosError) as ei:
        ctx.dos_kpm_moments(A, -9.6, 9.6, 10, 16, seed=5, precision="f64",
                            launch={"staged": 4}, flags=dos.DOS_OPT_TEST_STALL_WAIT,
                            wait_limit_cycles=2_000_000)
    assert ei.value.status == dos.DOS_ETIMEOUT
    mu = ctx.dos_kpm_moments(A, -9.6, 9.6, 10, 16, seed=5, precision="f64", launch={"staged": 4})
    ref = okpm.kpm_moments(anderson_3d(8, 6.0, seed=4), -9.6, 9.6, 10, 16, seed=5)
    assert np.abs(mu - ref).max() < TOL64


def test_unknown_variant_is_rejected(ctx):
    from paper_1308_5467_gb300 import dos
    A = anderson_3d(6, 6.0, seed=4)
    for launch in ({"staged": 5}, {"staged": 3, "depth": 3}, {"staged": 3, "depth": 16},
                   {"staged": 4, "depth": 4}, {"staged": 1, "depth": 4}, {"depth": 4}):
        with pytest.raises(dos.DosError):
            ctx.dos_kpm_moments(dev(A), -9.6, 9.6, 10, 16, seed=5, precision="f64",
                                launch=launch)


def test_wide_chunks_need_whole_32_byte_rows(ctx):
    from paper_1308_5467_gb300 import dos
    A = anderson_3d(6, 6.0, seed=4)
    with pytest.raises(dos.DosError):       # FP32, n_v = 20 -> rows of 80 bytes
        ctx.dos_kpm_moments(dev(A.astype(np.float32)), -9.6, 9.6, 10, 20, seed=5,
                            precision="f32", launch={"chunk_bytes": 32})
    with pytest.raises(dos.DosError):       # only with direct loads
        ctx.dos_kpm_moments(dev(A), -9.6, 9.6, 10, 16, seed=5, precision="f64",
                            launch={"chunk_bytes": 32, "staged": 2})


def test_bounded_wait_timeout_is_reported_and_context_survives(ctx):
    """Failure detection: the staged kernel's wait is made to run out (it
    expects bytes that never arrive); the call returns DOS_ETIMEOUT after the
    short limit and the next call on the same context works."""
    from paper_1308_5467_gb300 import dos
    A = dev(anderson_3d(10, 3.0, seed=2))
    with pytest.raises(dos.DosError) as ei:
        ctx.dos_kpm_moments(A, -8.0, 8.0, 10, 16, seed=1, precision="f32",
                            launch={"staged": 2}, flags=dos.DOS_OPT_TEST_STALL_WAIT,
                            wait_limit_cycles=2_000_000)
    assert ei.value.status == dos.DOS_ETIMEOUT
    ok = ctx.dos_kpm_moments(A, -8.0, 8.0, 10, 16, seed=1, precision="f32",
                             launch={"staged": 2})
    ref = okpm.kpm_moments(anderson_3d(10, 3.0, seed=2).astype(np.float32), -8.0, 8.0, 10, 16,
                           seed=1)
    assert np.all(np.abs(ok - ref) <= tol32(10, 1000 * 16))


def test_launch_shape_that_misses_columns_is_rejected(ctx):
    from paper_1308_5467_gb300 import dos
    A = anderson_3d(5, 1.0, seed=3)
    with pytest.raises(dos.DosError) as ei:  # 4 x 4 chunks of 2 doubles < 64 columns
        ctx.dos_kpm_moments(dev(A), -8.0, 8.0, 10, 64, seed=5, precision="f64",
                            launch={"team": 4, "chunks": 4})
    assert ei.value.status == dos.DOS_EINVAL


def test_spectrum_escape_is_reported(ctx):
    from paper_1308_5467_gb300 import dos
    A = laplacian_2d(20)
    with pytest.raises(dos.DosError) as ei:
        ctx.dos_kpm_moments(dev(A), 0.5, 7.0, 60, 4, seed=1, precision="f64")
    assert ei.value.status == dos.DOS_ESPECTRUM


def test_bad_inputs_are_rejected(ctx):
    import torch
    from paper_1308_5467_gb300 import dos
    A = laplacian_2d(6)
    with pytest.raises(dos.DosError) as ei:
        ctx.dos_kpm_moments(dev(A), 1.0, 1.0, 10, 4, seed=1)
    assert ei.value.status == dos.DOS_EINVAL
    bad = dos.CSRArrays(A.n, torch.from_numpy(A.row_ptr).cuda(),
                        torch.from_numpy(np.where(np.arange(A.nnz) == 5, 99, A.col_idx)
                                         .astype(np.int32)).cuda(),
                        torch.from_numpy(A.val).cuda())
    with pytest.raises(dos.DosError) as ei:
        ctx.dos_kpm_moments(bad, -0.1, 8.1, 10, 4, seed=1)
    assert ei.value.status == dos.DOS_EINVAL
    rp = A.row_ptr.copy()
    rp[3], rp[4] = rp[4], rp[3]
    bad2 = dos.CSRArrays(A.n, rp, A.col_idx, A.val)
    with pytest.raises(dos.DosError) as ei:
        ctx.dos_kpm_moments(bad2, -0.1, 8.1, 10, 4, seed=1)
    assert ei.value.status == dos.DOS_EINVAL
    with pytest.raises(dos.DosError) as ei:  # FP64 sweep of FP32 values
        ctx.dos_kpm_moments(dev(A, np.float32), -0.1, 8.1, 10, 4, seed=1, precision="f64")
    assert ei.value.status == dos.DOS_EINVAL


def test_graph_replay_matches_direct_launches(ctx):
    """Identical repeated calls are captured in a CUDA graph and replayed; the
    results equal those of kernel-by-kernel launches bit for bit."""
    from paper_1308_5467_gb300 import dos
    A = dev(anderson_3d(11, 5.0, seed=8))
    runs = [ctx.dos_kpm_moments(A, -9.0, 9.0, 90, 24, seed=6, precision="f32") for _ in range(4)]
    direct = ctx.dos_kpm_moments(A, -9.0, 9.0, 90, 24, seed=6, precision="f32",
                                 flags=dos.DOS_OPT_NO_GRAPH)
    for r in runs:
        assert np.array_equal(r, direct)


@pytest.mark.parametrize("launch", [None, {"team": 4, "chunks": 2, "chunk_bytes": 32},
                                    {"staged": 2}])
def test_dependent_launch_matches_plain_stream_order(ctx, launch):
    """Programmatic dependent launch between sweep steps changes when blocks are
    scheduled, not what they compute: bitwise equal to plain stream order, with
    and without graph capture."""
    from paper_1308_5467_gb300 import dos
    A = dev(anderson_3d(11, 5.0, seed=8).astype(np.float32))
    kw = dict(precision="f32", launch=launch)
    ref = ctx.dos_kpm_moments(A, -9.0, 9.0, 90, 64, 6, flags=dos.DOS_OPT_NO_PDL | dos.DOS_OPT_NO_GRAPH,
                              **kw)
    for flags in (0, dos.DOS_OPT_NO_GRAPH, dos.DOS_OPT_NO_PDL):
        for _ in range(3):                    # the third identical call replays a graph
            assert np.array_equal(ctx.dos_kpm_moments(A, -9.0, 9.0, 90, 64, 6, flags=flags, **kw),
                                  ref)


def test_profiling_counts_step_launches(ctx):
    A = dev(laplacian_2d(30))
    ctx.dos_profile_enable(True)
    ctx.dos_kpm_moments(A, -0.1, 8.1, 41, 8, seed=1, precision="f64")
    prof = ctx.dos_profile_read()
    ctx.dos_profile_enable(False)
    assert prof["step_launches"] == 21 and prof["sweeps"] == 1
    assert prof["step_ms"] > 0 and prof["launches"] >= 21
