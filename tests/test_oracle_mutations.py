"""The pins must catch plausible mistakes.  Each test plants one mistake in a
copy of the oracle (on the CPU) and checks that the pin it targets fails:

* the doubling identity with the sign the paper prints (Appendix A: "+");
* the shift c dropped from B = (A - cI)/d;
* the factor 2 of the k >= 1 terms dropped from the reconstruction;
* the Jackson factor with cos and sin swapped.
"""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

from oracle import dos as odos
from oracle import kpm as okpm
from synthetic import random_symmetric

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                   "kpm_oracle.c")


def build_mutant(tmp_path, old: str, new: str) -> C.CDLL:
    text = open(SRC).read()
    assert old in text, old
    mutant = tmp_path / "mutant.c"
    mutant.write_text(text.replace(old, new, 1))
    so = tmp_path / "mutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", str(so), str(mutant),
                    "-lm"], check=True)
    lib = C.CDLL(str(so))
    lib.oracle_kpm_moments.restype = C.c_int
    lib.oracle_kpm_moments.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                                       C.c_double, C.c_int, C.c_int64, C.c_int64, C.c_uint64,
                                       C.c_uint64, C.c_int, C.c_int, C.c_int, C.c_void_p]
    return lib


def eig_pin_residual(lib, mode):
    """max |oracle - exact| of the dense-eigendecomposition pin."""
    A = random_symmetric(60, 0.1, 1, empty_rows=2)
    lam, U = np.linalg.eigh(A.to_dense())
    lb, ub = lam[0] - 0.3, lam[-1] + 0.2
    c, d = 0.5 * (lb + ub), 0.5 * (ub - lb)
    M, nv = 37, 3
    out = np.empty((nv, M + 1))
    rp, ci, va = okpm._csr_arrays(A.row_ptr, A.col_idx, A.val)
    rc = lib.oracle_kpm_moments(A.n, rp.ctypes.data, ci.ctypes.data, va.ctypes.data, lb, ub, M,
                                nv, 0, 11, 0, mode, 0, 1, out.ctypes.data)
    assert rc == 0
    V = okpm.start_block(A.n, nv, seed=11)
    worst = 0.0
    for l in range(nv):
        w = (U.T @ V[:, l]) ** 2 / A.n
        t = (lam - c) / d
        exact = np.array([np.sum(w * np.cos(k * np.arccos(np.clip(t, -1, 1)))) for k in range(M + 1)])
        worst = max(worst, np.abs(out[l] - exact).max())
    return worst


def test_unmutated_copy_passes(tmp_path):
    lib = build_mutant(tmp_path, "- mu[1];", "- mu[1];")
    assert eig_pin_residual(lib, 1) < 1e-12


def test_paper_sign_of_doubling_is_caught(tmp_path):
    lib = build_mutant(tmp_path, "/ dn - mu[1];", "/ dn + mu[1];")
    assert eig_pin_residual(lib, 1) > 1e-3


def test_dropped_shift_is_caught(tmp_path):
    lib = build_mutant(tmp_path, "y[i] = (y[i] - c * x[i]) / d;", "y[i] = y[i] / d;")
    assert eig_pin_residual(lib, 0) > 1e-3
    assert eig_pin_residual(lib, 1) > 1e-3


def orthogonality_residual():
    rng = np.random.default_rng(1)
    M, N = 40, 200
    mu = np.concatenate([[1.0], rng.uniform(-0.5, 0.5, M)])
    t, phi, _ = odos.reconstruct(mu, "none", N_t=N)
    w = np.pi / N * np.sqrt(1 - t * t) * phi
    return max(abs(np.sum(w * np.cos(j * np.arccos(t))) - mu[j]) for j in range(M + 1))


def test_dropped_factor_two_is_caught(monkeypatch):
    assert orthogonality_residual() < 1e-12

    def poly_without_two(mu, g, t):
        k = np.arange(mu.shape[0])
        T = np.cos(np.outer(np.arccos(np.clip(t, -1.0, 1.0)), k))
        return T @ (g * mu)
    monkeypatch.setattr(odos, "_poly", poly_without_two)
    assert orthogonality_residual() > 1e-2


def test_swapped_jackson_terms_are_caught(monkeypatch):
    import math

    def bad_jackson(M):
        a = math.pi / (M + 2)
        k = np.arange(M + 1, dtype=np.float64)
        return ((1.0 - k / (M + 2)) * math.sin(a) * np.sin(k * a)
                + (1.0 / (M + 2)) * math.cos(a) * np.cos(k * a)) / math.sin(a)
    monkeypatch.setattr(odos, "jackson", bad_jackson)
    g = odos.jackson(30)
    mu = np.cos(np.arange(31) * np.arccos(0.3))
    _, pj, _ = odos.reconstruct(mu, "jackson", t=np.linspace(-0.99, 0.99, 999))
    with pytest.raises(AssertionError):
        assert abs(g[0] - 1.0) < 1e-15 and pj.min() >= -1e-12 * pj.max()


def legendre_pin_residual(lib):
    """max |oracle - exact| of the dense-eig pin of the Legendre moments (mode 2)."""
    import scipy.special
    A = random_symmetric(60, 0.1, 1, empty_rows=2)
    lam, U = np.linalg.eigh(A.to_dense())
    lb, ub = lam[0] - 0.3, lam[-1] + 0.2
    c, d = 0.5 * (lb + ub), 0.5 * (ub - lb)
    M, nv = 30, 2
    out = np.empty((nv, M + 1))
    rp, ci, va = okpm._csr_arrays(A.row_ptr, A.col_idx, A.val)
    assert lib.oracle_kpm_moments(A.n, rp.ctypes.data, ci.ctypes.data, va.ctypes.data, lb, ub,
                                  M, nv, 0, 5, 0, 2, 0, 1, out.ctypes.data) == 0
    W = (U.T @ okpm.start_block(A.n, nv, seed=5)) ** 2 / A.n
    Lk = np.array([scipy.special.eval_legendre(k, (lam - c) / d) for k in range(M + 1)])
    return np.abs(out - (Lk @ W).T).max()


def test_legendre_recurrence_coefficient_is_caught(tmp_path):
    (tmp_path / "good").mkdir()
    (tmp_path / "bad").mkdir()
    good = build_mutant(tmp_path / "good", "(2.0 * k + 1.0) / (k + 1.0)",
                        "(2.0 * k + 1.0) / (k + 1.0)")
    assert legendre_pin_residual(good) < 1e-12
    bad = build_mutant(tmp_path / "bad", "(2.0 * k + 1.0) / (k + 1.0)", "(2.0 * k) / (k + 1.0)")
    assert legendre_pin_residual(bad) > 1e-3


def test_dgl_boundary_term_sign_is_caught():
    """Flip the parity sign of zeta_k (Eq. eta) in a copy of the DGL oracle; the
    quadrature pin of Eq. DGLcoeff must fail."""
    import types

    import scipy.special
    from oracle import legendre as oleg
    text = open(oleg.__file__).read()
    old = "zeta = e_plus - (e_minus if k % 2 == 0 else -e_minus)"
    assert old in text
    mod = types.ModuleType("oracle.legendre_mutant")
    mod.__package__ = "oracle"
    exec(compile(text.replace(old, "zeta = e_plus + (e_minus if k % 2 == 0 else -e_minus)"),
                 "legendre_mutant", "exec"), mod.__dict__)
    s, w = scipy.special.roots_legendre(2000)
    t, sigma = 0.1, 0.5                      # wide, so both boundary terms matter
    G = np.exp(-0.5 * ((s - t) / sigma) ** 2)
    for m, expect_ok in ((oleg, True), (mod, False)):
        g = m.dgl_gamma(t, sigma, 200)
        ref = np.array([np.sum(w * scipy.special.eval_legendre(k, s) * G) for k in range(g.shape[0])])
        assert (np.abs(g - ref).max() < 1e-10) == expect_ok
