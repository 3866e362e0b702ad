"""Config 3: normalized Laplacian of a Chung-Lu graph (beta = 2.5, mean degree
20, skewed rows up to ~10^4 nonzeros), FP32 form, M = 1000, n_v = 256, in the
launch configuration the benchmark times (the autotuner's choice, whose
moments are the totals over the vectors) and with the bounds it uses: [0, 2],
the interval that holds the spectrum of every normalized Laplacian, padded by
1% of the width per side.  This graph reaches both ends -- 726 isolated
vertices (eigenvalue 0) and an isolated edge (eigenvalue 2, weight 2/n) -- so
the interval is tight, and no Lanczos run from a random vector can be relied
on to see the isolated edge: 20 steps return an upper bound near 1.6.

The oracle cannot sweep 256 vectors of 4.2 M rows to degree 1000 inside a test,
so the tuned kernel instance is checked three ways:
* all 256 vectors at full size: properties that hold at any size (mu_0 = 1,
  |mu_k| <= 1, Jackson DOS >= 0 within the FP32 slack) and the totals equal to
  the mean of the per-vector moments of the per-vector instance;
* the same instance (the tuned launch shape forced) on a panel of 4 vectors at
  vector offset 100 of the full-size graph, totals only, against the oracle
  over those 4 vectors, element by element for k <= 200;
* the same instance on the same recipe at n = 262,144, a panel of 8 vectors,
  against the oracle element by element for every k <= M = 1000.
Tolerance: the FP32 bound of tests/tolerances.py.
"""
import os

import numpy as np
import pytest

from oracle import kpm as okpm
from synthetic import chung_lu_normalized_laplacian
from tolerances import fp32_ratio, tol32

pytestmark = pytest.mark.gpu

M, N_V = 1000, 256
CORES = os.cpu_count() or 1
BOUNDS = (-0.02, 2.02)


@pytest.fixture(scope="module")
def ctx():
    from paper_1308_5467_gb300 import dos
    c = dos.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def graph():
    return chung_lu_normalized_laplacian(4194304, beta=2.5, mean_deg=20.0, seed=3).astype(
        np.float32)


@pytest.fixture(scope="module")
def tuned(ctx, graph):
    """Device copy, bounds and launch shape exactly as the benchmark makes them."""
    from paper_1308_5467_gb300 import dos
    Ad = dos.CSRArrays.from_synthetic(graph, device="cuda")
    lb, ub = BOUNDS
    shape, _ = ctx.dos_tune(Ad, N_V, "f32")
    return Ad, lb, ub, shape


def test_graph_reaches_both_ends_of_the_interval(graph):
    """Eigenvalue 0 (isolated vertices: a stored zero diagonal, row length 1) and
    eigenvalue 2 (an isolated edge: two rows of degree 1 joined to each other), so
    no interval narrower than [0, 2] encloses the spectrum."""
    deg = np.diff(graph.row_ptr) - 1
    assert np.any(deg == 0)
    rows = np.repeat(np.arange(graph.n), np.diff(graph.row_ptr))
    off = graph.col_idx != rows
    assert np.any((deg[rows[off]] == 1) & (deg[graph.col_idx[off]] == 1))


def test_full_size_all_vectors(ctx, graph, tuned):
    Ad, lb, ub, shape = tuned
    assert graph.meta["max_row_len"] > 2000  # skewed rows are present
    mu = ctx.dos_kpm_moments(Ad, lb, ub, M, N_V, seed=3, precision="f32")
    assert mu[0] == 1.0 and np.all(np.abs(mu) <= 1.0 + 1e-6)
    pv = np.empty((N_V, M + 1))
    mu_pv = ctx.dos_kpm_moments(Ad, lb, ub, M, N_V, seed=3, precision="f32", mu_per_vec=pv)
    assert np.abs(pv.mean(axis=0) - mu_pv).max() < 1e-12
    # the totals-only and per-vector instances differ only in where the FP32 row
    # sums enter the float-pair accumulators
    assert np.abs(mu - mu_pv).max() < 1e-9
    # With exact moments P(t) = pi sqrt(1-t^2) phi_hat(t) = g_0 mu_0 + 2 sum g_k mu_k T_k(t)
    # is >= 0 (Jackson kernel, positive measure); the FP32 form may move it by at most
    # sum_k (2 - delta_k0) g_k |dmu_k| with |dmu_k| within the FP32 bound.
    from oracle.dos import chebyshev_nodes, jackson
    phi = ctx.dos_reconstruct(mu, M, "jackson", lb, ub, N_t=2000)
    t = chebyshev_nodes(2000)
    P = np.pi * np.sqrt(1 - t * t) * phi
    slack = np.sum(np.where(np.arange(M + 1) == 0, 1.0, 2.0) * jackson(M) *
                   tol32(M, graph.n * N_V))
    assert P.min() >= -slack


def test_full_size_tuned_instance_panel_vs_oracle(ctx, graph, tuned):
    Ad, lb, ub, shape = tuned
    K, nv, off = 200, 4, 100
    mu = ctx.dos_kpm_moments(Ad, lb, ub, K, nv, seed=3, precision="f32", vec_offset=off,
                             launch=shape)
    ref = okpm.kpm_moments(graph, lb, ub, K, nv, seed=3, vec_offset=off,
                           nthreads=min(CORES, nv))
    print("tuned", shape, "panel ratio to u sqrt(k+1):", fp32_ratio(mu, ref))
    assert np.all(np.abs(mu - ref) <= tol32(K, graph.n * nv)), fp32_ratio(mu, ref)


def test_quarter_million_rows_tuned_instance_every_k(ctx, tuned):
    from paper_1308_5467_gb300 import dos
    _, _, _, shape = tuned
    A = chung_lu_normalized_laplacian(262144, beta=2.5, mean_deg=20.0, seed=3).astype(
        np.float32)
    Ad = dos.CSRArrays.from_synthetic(A, device="cuda")
    lb, ub = BOUNDS
    nv, off = 8, 37
    launch = {k: v for k, v in shape.items() if k != "tiles"}  # tiles sized for this n
    mu = ctx.dos_kpm_moments(Ad, lb, ub, M, nv, seed=3, precision="f32", vec_offset=off,
                             launch=launch)
    ref = okpm.kpm_moments(A, lb, ub, M, nv, seed=3, vec_offset=off, nthreads=min(CORES, nv))
    print("262k ratio to u sqrt(k+1):", fp32_ratio(mu, ref))
    assert np.all(np.abs(mu - ref) <= tol32(M, A.n * nv)), fp32_ratio(mu, ref)
