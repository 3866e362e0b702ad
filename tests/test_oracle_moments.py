"""Pins of the oracle's moment sweep against facts fixed outside the oracle.

Each test compares oracle.kpm with a result the paper or the mathematics fixes:
the published splitmix64 outputs, dense eigendecompositions (Theorem 3.1 and
Eq. expmu make the estimate an exact weighted sum over eigenvalues for fixed
vectors), the closed-form spectra of the Dirichlet Laplacian and the clean
periodic lattice, the diagonal special case and the Chebyshev invariants.
"""
import math

import numpy as np
import pytest
import scipy.fft

from oracle import kpm
from synthetic import anderson_3d, diagonal, laplacian_2d, random_symmetric


def cheb_T(k, x):
    return np.cos(k * np.arccos(np.clip(x, -1.0, 1.0)))


def weighted_moments(lam_hat, weights, M):
    """sum_j w_j T_k(lam_hat_j) for k = 0..M (weights already include 1/n)."""
    return np.array([np.sum(weights * cheb_T(k, lam_hat)) for k in range(M + 1)])


# ---- the random start vectors ------------------------------------------------

def test_splitmix64_published_outputs():
    # Reference outputs of splitmix64 seeded with 0 (Steele, Lea, Flood 2014;
    # the published C reference implementation).
    assert kpm.splitmix64_stream(0, 3) == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                           0x06C45D188009454F]


@pytest.mark.parametrize("seed", [0, 12345, 2**63 + 17])
def test_rademacher_is_bit_of_stream_word(seed):
    # Entry (b=0, l, i) is bit l of stream output number i+1 (l < 64).
    words = kpm.splitmix64_stream(seed, 4)
    for i in range(4):
        for l in (0, 1, 31, 63):
            bit = (words[i] >> l) & 1
            assert kpm.rademacher(seed, 0, l, i) == (-1.0 if bit else 1.0)


def test_rademacher_counter_fields_distinct():
    # (b, floor(l/64), i) select distinct words: blocks must not repeat.
    a = kpm.start_block(4096, 128, seed=7, batch_index=0)
    b = kpm.start_block(4096, 128, seed=7, batch_index=1)
    assert not np.array_equal(a, b)
    assert not np.array_equal(a[:, :64], a[:, 64:])


def test_rademacher_moments_condition():
    # E[v] = 0 and E[v v^T] = I (Theorem 3.1's condition), within 5 sigma.
    n, nv = 20000, 32
    V = kpm.start_block(n, nv, seed=3)
    assert set(np.unique(V)) == {-1.0, 1.0}
    assert np.all(np.abs(V.mean(axis=0)) < 5.0 / math.sqrt(n))
    G = V.T @ V / n
    off = G - np.diag(np.diag(G))
    assert np.allclose(np.diag(G), 1.0)
    assert np.abs(off).max() < 5.0 / math.sqrt(n)


# ---- moments vs dense eigendecomposition -------------------------------------

@pytest.mark.parametrize("mode", ["direct", "doubling"])
@pytest.mark.parametrize("n,density,seed,M", [(60, 0.1, 1, 37), (150, 0.04, 2, 80),
                                               (97, 0.2, 3, 101)])
def test_moments_match_dense_eig(mode, n, density, seed, M):
    A = random_symmetric(n, density, seed, empty_rows=2)
    D = A.to_dense()
    lam, U = np.linalg.eigh(D)
    lb, ub = lam[0] - 0.3, lam[-1] + 0.2
    c, d = 0.5 * (lb + ub), 0.5 * (ub - lb)
    nv = 3
    V = kpm.start_block(n, nv, seed=11)
    mu_pv = kpm.kpm_moments_per_vector(A, lb, ub, M, nv, seed=11, mode=mode)
    for l in range(nv):
        w = (U.T @ V[:, l]) ** 2 / n
        exact = weighted_moments((lam - c) / d, w, M)
        assert np.abs(mu_pv[l] - exact).max() < 1e-12


def test_direct_and_doubling_agree_and_invariants():
    A = laplacian_2d(20)
    mu_d = kpm.kpm_moments_per_vector(A, -0.08, 8.08, 150, 5, seed=1, mode="direct")
    mu_2 = kpm.kpm_moments_per_vector(A, -0.08, 8.08, 150, 5, seed=1, mode="doubling")
    assert np.abs(mu_d - mu_2).max() < 1e-12
    assert np.all(mu_2[:, 0] == 1.0)          # v^T v / n = 1 exactly for +-1 entries
    assert np.abs(mu_2).max() <= 1.0 + 1e-12  # weighted average of T_k on [-1, 1]


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_low_degree_modes(M):
    A = random_symmetric(30, 0.2, 5)
    lam = np.linalg.eigvalsh(A.to_dense())
    lb, ub = lam[0] - 0.1, lam[-1] + 0.1
    a = kpm.kpm_moments_per_vector(A, lb, ub, M, 2, seed=4, mode="direct")
    b = kpm.kpm_moments_per_vector(A, lb, ub, M, 2, seed=4, mode="doubling")
    assert a.shape == (2, M + 1)
    assert np.abs(a - b).max() < 1e-13


# ---- closed forms ------------------------------------------------------------

def laplacian_exact_weights(m, v):
    """Eigenvalues and the weights (u_ij^T v)^2 / n of the m x m Dirichlet
    Laplacian, with u_ij(a, b) = (2/(m+1)) sin(i a pi/(m+1)) sin(j b pi/(m+1))."""
    i = np.arange(1, m + 1)
    lam = (4.0 - 2.0 * np.cos(i[:, None] * np.pi / (m + 1))
           - 2.0 * np.cos(i[None, :] * np.pi / (m + 1)))
    # DST-I along both axes: y_k = 2 sum_n x_n sin(pi (k+1)(n+1)/(N+1)).
    beta = scipy.fft.dstn(v.reshape(m, m), type=1) * (2.0 / (m + 1)) / 4.0
    return lam.ravel(), (beta ** 2).ravel() / (m * m)


def test_laplacian_40x40_closed_form():
    m = 40
    A = laplacian_2d(m)
    lb, ub = -0.08, 8.08
    c, d = 0.5 * (lb + ub), 0.5 * (ub - lb)
    M, nv = 100, 20
    V = kpm.start_block(m * m, nv, seed=1)
    mu_pv = kpm.kpm_moments_per_vector(A, lb, ub, M, nv, seed=1, mode="doubling")
    for l in range(nv):
        lam, w = laplacian_exact_weights(m, V[:, l])
        assert abs(w.sum() - 1.0) < 1e-13          # Parseval: the modes are orthonormal
        exact = weighted_moments((lam - c) / d, w, M)
        assert np.abs(mu_pv[l] - exact).max() < 1e-12
    # Stochastic estimate of the trace moments (1/n) sum_j T_k(lam_j):
    # Rademacher variance per vector <= 2, so the std of the mean is <= sqrt(2/(n n_v)).
    lam, _ = laplacian_exact_weights(m, V[:, 0])
    trace = np.array([cheb_T(k, (lam - c) / d).mean() for k in range(M + 1)])
    assert np.abs(mu_pv.mean(axis=0) - trace).max() < 5.0 * math.sqrt(2.0 / (m * m * nv))


def test_clean_periodic_lattice_fft():
    L = 8
    A = anderson_3d(L, 0.0, seed=0)
    n = L ** 3
    q = 2.0 * np.pi * np.arange(L) / L
    lam = -2.0 * (np.cos(q)[:, None, None] + np.cos(q)[None, :, None] + np.cos(q)[None, None, :])
    lb, ub = -6.06, 6.06
    c, d = 0.0, 6.06
    M, nv = 64, 4
    V = kpm.start_block(n, nv, seed=9)
    mu_pv = kpm.kpm_moments_per_vector(A, lb, ub, M, nv, seed=9, mode="doubling")
    for l in range(nv):
        vh = np.fft.fftn(V[:, l].reshape(L, L, L))
        w = (np.abs(vh) ** 2 / n).ravel() / n
        exact = weighted_moments((lam.ravel() - c) / d, w, M)
        assert np.abs(mu_pv[l] - exact).max() < 1e-12


def test_diagonal_matrix_is_exact_for_any_vectors():
    rng = np.random.default_rng(0)
    dvals = rng.uniform(-3.0, 5.0, size=257)
    A = diagonal(dvals)
    lb, ub = -3.5, 5.5
    c, d = 0.5 * (lb + ub), 0.5 * (ub - lb)
    M = 90
    exact = np.array([cheb_T(k, (dvals - c) / d).mean() for k in range(M + 1)])
    for seed in (0, 1, 99):
        for mode in ("direct", "doubling"):
            mu = kpm.kpm_moments(A, lb, ub, M, 6, seed=seed, mode=mode)
            assert np.abs(mu - exact).max() < 1e-13


def test_vector_offset_shards_concatenate():
    # Start vectors l in [off, off+k) of one run equal a run shifted by off.
    A = laplacian_2d(12)
    full = kpm.kpm_moments_per_vector(A, -0.1, 8.1, 30, 8, seed=5)
    part = kpm.kpm_moments_per_vector(A, -0.1, 8.1, 30, 3, seed=5, vec_offset=5)
    assert np.array_equal(full[5:8], part)


def test_rounding_order_spread_is_small():
    # Headroom for the GPU tolerance: reversing the summation order of every
    # dot product moves the FP64 moments by far less than 1e-12.
    A = anderson_3d(12, 4.0, seed=2)
    lb, ub = -10.2, 10.2
    a = kpm.kpm_moments(A, lb, ub, 200, 4, seed=2, reverse=False)
    b = kpm.kpm_moments(A, lb, ub, 200, 4, seed=2, reverse=True)
    assert np.abs(a - b).max() < 1e-13
