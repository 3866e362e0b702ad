"""The FP32 form's stated parity bound (tests/tolerances.py) checked on the
CPU against what it is meant to separate, on the benchmark inputs: the 64^3
Anderson lattice at full size and the power-law Chung-Lu recipe at 262,144
rows (the 4.2 M-row graph is too large for a CPU test).

An emulation of the form -- FP32 values, vectors and SpMM (scipy, FP32
accumulation), the step's shift and scale with c and 1/d as float pairs,
dot products of the FP32 vectors in FP64 -- stays within the bound, and the
same emulation with the dot products accumulated over the rows in plain FP32
exceeds it many times over, so a kernel whose accumulator degraded to FP32
would fail the GPU parity tests.  Both are compared with the FP64 oracle on
the same FP32-rounded values and start vectors."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import kpm as okpm
from synthetic import anderson_3d, chung_lu_normalized_laplacian
from tolerances import U32, tol32


def emulate(A, lb, ub, M, n_v, seed, fp32_dots):
    A32 = sp.csr_matrix((A.val.astype(np.float32), A.col_idx, A.row_ptr), shape=(A.n, A.n))
    X0 = okpm.start_block(A.n, n_v, seed).astype(np.float32)
    c, s = 0.5 * (lb + ub), 1.0 / (0.5 * (ub - lb))
    chi, shi = np.float32(c), np.float32(s)
    clo, slo = np.float32(c - float(chi)), np.float32(s - float(shi))

    def apply(X):
        t = (A32 @ X - chi * X) - clo * X
        return t * shi + t * slo

    def dot(a, b):
        if fp32_dots:  # one FP32 accumulator per vector, running down the rows
            return np.cumsum((a * b).astype(np.float32), axis=0, dtype=np.float32)[-1] \
                .astype(np.float64)
        return np.einsum("ij,ij->j", a.astype(np.float64), b.astype(np.float64))

    n = A.n
    mu = np.zeros((n_v, M + 1))
    Xp, Xc = X0, apply(X0)
    mu[:, 0] = dot(X0, X0) / n
    mu[:, 1] = dot(Xc, X0) / n
    mu[:, 2] = 2 * dot(Xc, Xc) / n - mu[:, 0]
    for k in range(1, (M + 1) // 2):
        Xn = np.float32(2) * apply(Xc) - Xp
        if 2 * k + 1 <= M:
            mu[:, 2 * k + 1] = 2 * dot(Xn, Xc) / n - mu[:, 1]
        if 2 * k + 2 <= M:
            mu[:, 2 * k + 2] = 2 * dot(Xn, Xn) / n - mu[:, 0]
        Xp, Xc = Xc, Xn
    return mu


@pytest.mark.parametrize("name", ["anderson64", "chunglu262k"])
def test_bound_separates_fp32_vectors_from_fp32_accumulation(name):
    if name == "anderson64":
        A = anderson_3d(64, 4.0, seed=2).astype(np.float32)
        lb, ub, M = -8.16, 8.16, 200
    else:
        A = chung_lu_normalized_laplacian(262144, 2.5, 20.0, seed=3).astype(np.float32)
        lb, ub, M = -0.02, 2.02, 400
    n_v, seed = 4, 2
    ref = okpm.kpm_moments_per_vector(A, lb, ub, M, n_v, seed)
    bound = tol32(M, A.n)                       # per-vector moments: N = n
    k = np.arange(M + 1)
    good = np.abs(emulate(A, lb, ub, M, n_v, seed, False) - ref)
    bad = np.abs(emulate(A, lb, ub, M, n_v, seed, True) - ref)
    print(name, "FP32 vectors: %.3f of the bound; FP32 accumulation: %.0f x the bound, "
          "%.0f u sqrt(k+1)" % ((good / bound).max(), (bad / bound).max(),
                                (bad / (U32 * np.sqrt(k + 1))).max()))
    assert np.all(good <= 0.5 * bound)
    assert (bad / bound).max() > 50
