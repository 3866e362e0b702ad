"""Config 3 at full size: normalized Laplacian of a Chung-Lu graph (n =
4,194,304, beta = 2.5, mean degree 20, skewed rows up to ~10^4 nonzeros),
M = 1000, n_v = 256, FP32 SpMM.  The oracle cannot sweep 256 vectors of this
size in a test, so sampled vectors are checked one by one (their moments up to
k = 200, which do not depend on M), and properties that hold at any size are
checked for all moments: mu_0 = 1, |mu_k| <= 1, Jackson DOS >= 0."""
import os

import numpy as np
import pytest

from oracle import kpm as okpm
from synthetic import chung_lu_normalized_laplacian

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def graph():
    return chung_lu_normalized_laplacian(4194304, beta=2.5, mean_deg=20.0, seed=3)


def test_chung_lu_full_size_sampled(graph):
    from paper_1308_5467_gb300 import dos
    A = graph.astype(np.float32)
    assert A.meta["max_row_len"] > 2000  # skewed rows are present
    lb, ub = -0.02, 2.02                  # the spectrum of I - D^-1/2 A D^-1/2 lies in [0, 2]
    M, n_v = 1000, 256
    with dos.Context(0) as ctx:
        Ad = dos.CSRArrays.from_synthetic(A, device="cuda")
        ctx.dos_tune(Ad, n_v, "f32")      # the launch configuration the benchmark times
        pv = np.empty((n_v, M + 1))
        mu = ctx.dos_kpm_moments(Ad, lb, ub, M, n_v, seed=3, precision="f32", mu_per_vec=pv)
        phi = ctx.dos_reconstruct(mu, M, "jackson", lb, ub, N_t=2000)
    assert mu[0] == 1.0 and np.all(np.abs(mu) <= 1.0 + 1e-4)
    assert np.abs(pv.mean(axis=0) - mu).max() < 1e-9
    # With exact moments P(t) = pi sqrt(1-t^2) phi_hat(t) = g_0 mu_0 + 2 sum g_k mu_k T_k(t)
    # is >= 0 (Jackson kernel, positive measure); the FP32 form may move it by at most
    # sum_k (2 - delta_k0) g_k |dmu_k| with |dmu_k| within the stated FP32 bound.
    from oracle.dos import chebyshev_nodes, jackson
    t = chebyshev_nodes(2000)
    P = np.pi * np.sqrt(1 - t * t) * phi
    tolk = 2e-7 * (np.arange(M + 1) + 1) + 1e-6
    slack = np.sum(np.where(np.arange(M + 1) == 0, 1.0, 2.0) * jackson(M) * tolk)
    assert P.min() >= -slack
    K = 200
    picks = [0, 255]
    ref = okpm.kpm_moments_per_vector(A, lb, ub, K, 1, seed=3, vec_offset=picks[0],
                                      nthreads=os.cpu_count() or 1)
    ref2 = okpm.kpm_moments_per_vector(A, lb, ub, K, 1, seed=3, vec_offset=picks[1],
                                       nthreads=os.cpu_count() or 1)
    tol = 2e-7 * (np.arange(K + 1) + 1) + 1e-6
    assert np.all(np.abs(pv[picks[0], :K + 1] - ref[0]) <= tol)
    assert np.all(np.abs(pv[picks[1], :K + 1] - ref2[0]) <= tol)
