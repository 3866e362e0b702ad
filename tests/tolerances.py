"""Tolerances of the GPU parity tests and the error model behind each.

FP64 form: 1e-12 absolute per moment (the moments are O(1), mu_0 = 1).  The
GPU and the oracle run the same recurrence in FP64 and differ only in the
order of the additions of the SpMV rows and of the dot products; that spread
grows about like k^1.5 * 2^-53 and stays below 1e-13 at M = 1000.

FP32 form (FP32 values, vectors and SpMM; the dot products formed in FP32 per
row, carried as float pairs per thread and reduced in FP64), compared with
the FP64 oracle run on the same FP32-representable values:

    |mu_k(FP32 form) - mu_k(oracle)| <= u sqrt(k + 1) (1/2 + 40 / sqrt(N)),

u = 2^-24, N the number of (row, vector) terms the moment averages: n for a
per-vector moment, n n_v for the mean over n_v vectors.  At the benchmark
sizes (N >= 1.6e7) that is 0.5 u sqrt(k+1): 9.4e-7 at k = 1000.  The model:
the kernels apply B = (A - cI)/d with c and 1/d kept to about 2^-48, so the
one source of error is the rounding of every step's result X_{k+1} to FP32
(relative u per element).  A rounding made at step j reaches step k through
U_{k-1-j}(B), whose norm is at most 1/sin(theta) <= 5 once the bounds are
padded by 1% per side; the roundings of different steps have no common sign,
so the error of X_k grows like sqrt(k).  The moment error is the dot product
of X_k with that error over N terms: a random-sign part that shrinks like
20 u sqrt(k) / sqrt(N) (the second term), and a part that does not average
out, from roundings shared by rows with the same stencil values (the first).
Measured against it, in a CPU emulation of the form that reproduces the
kernels' results to 9 digits and on the GPU, every test matrix and workload
stays at or below 0.55 of the bound (the worst: a 9 x 9 Laplacian, n = 81,
per vector).  The bound catches a degraded accumulator: accumulating the dot
products over the rows in plain FP32 gives 330 - 17,000 u sqrt(k+1) on the
64^3 lattice and on power-law graphs (tests/test_fp32_error_model.py).
"""
import numpy as np

TOL64 = 1e-12
U32 = 2.0 ** -24


def tol32(M, N):
    """Per-moment bound of the FP32 form for k = 0..M (array of M+1); N = rows
    times vectors averaged by the moment (n per vector, n n_v for the mean)."""
    return U32 * np.sqrt(np.arange(M + 1) + 1.0) * (0.5 + 40.0 / np.sqrt(float(N)))


def fp32_ratio(mu, ref):
    """max_k |mu_k - ref_k| / (u sqrt(k+1)) over the last axis (any leading shape)."""
    mu, ref = np.asarray(mu), np.asarray(ref)
    k = np.arange(mu.shape[-1])
    return float((np.abs(mu - ref) / (U32 * np.sqrt(k + 1.0))).max())
