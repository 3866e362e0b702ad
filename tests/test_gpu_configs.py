"""Parity at the full sizes of the benchmark workload (3-D Anderson model,
64^3 periodic lattice, W = 4, M = 500, n_v = 64) in the launch configuration
the benchmark times, FP64 and FP32-SpMM forms, against the oracle run over all
64 vectors on the host cores."""
import os

import numpy as np
import pytest

from oracle import bounds as obounds
from oracle import kpm as okpm
from synthetic import anderson_3d
from tolerances import fp32_ratio, tol32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1308_5467_gb300 import dos
    c = dos.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def anderson64():
    return anderson_3d(64, 4.0, seed=2)


@pytest.fixture(scope="module")
def oracle_mu(anderson64):
    lb, ub = obounds.bounds(anderson64, "gershgorin", pad_frac=0.01)
    pv = okpm.kpm_moments_per_vector(anderson64, lb, ub, 500, 64, seed=2,
                                     nthreads=os.cpu_count() or 1)
    pv32 = okpm.kpm_moments_per_vector(anderson64.astype(np.float32), lb, ub, 500, 64, seed=2,
                                       nthreads=os.cpu_count() or 1)
    return lb, ub, pv, pv32


def test_bounds_gershgorin_exact(ctx, anderson64):
    from paper_1308_5467_gb300 import dos
    A = dos.CSRArrays.from_synthetic(anderson64, device="cuda")
    assert ctx.dos_bounds(A, "gershgorin", pad_frac=0.01) == \
        obounds.bounds(anderson64, "gershgorin", pad_frac=0.01)


def test_anderson64_f64_full(ctx, anderson64, oracle_mu):
    from paper_1308_5467_gb300 import dos
    lb, ub, pv_ref, _ = oracle_mu
    A = dos.CSRArrays.from_synthetic(anderson64, device="cuda")
    mu = ctx.dos_kpm_moments(A, lb, ub, 500, 64, seed=2, precision="f64")
    err = np.abs(mu - pv_ref.mean(axis=0))
    print("f64 max |dmu| =", err.max())
    assert err.max() < 1e-12
    # the launch configuration the benchmark times: the autotuner's choice, cached
    shape, _ = ctx.dos_tune(A, 64, "f64")
    mu_t = ctx.dos_kpm_moments(A, lb, ub, 500, 64, seed=2, precision="f64")
    print("f64 tuned", shape, "max |dmu| =", np.abs(mu_t - pv_ref.mean(axis=0)).max())
    assert np.abs(mu_t - pv_ref.mean(axis=0)).max() < 1e-12


def test_anderson64_f32_full(ctx, anderson64, oracle_mu):
    from paper_1308_5467_gb300 import dos
    lb, ub, pv64, pv32 = oracle_mu
    A = dos.CSRArrays.from_synthetic(anderson64, device="cuda", dtype=np.float32)
    bound = tol32(500, 262144 * 64)
    mu = ctx.dos_kpm_moments(A, lb, ub, 500, 64, seed=2, precision="f32")
    err = np.abs(mu - pv32.mean(axis=0))
    print("f32 max |dmu| =", err.max(), " vs f64 values:", np.abs(mu - pv64.mean(axis=0)).max(),
          " ratio to u sqrt(k+1):", fp32_ratio(mu, pv32.mean(axis=0)))
    assert np.all(err <= bound)
    # the launch configuration the benchmark times: the autotuner's choice, cached
    shape, _ = ctx.dos_tune(A, 64, "f32")
    mu_t = ctx.dos_kpm_moments(A, lb, ub, 500, 64, seed=2, precision="f32")
    print("f32 tuned", shape, "max |dmu| =", np.abs(mu_t - pv32.mean(axis=0)).max())
    assert np.all(np.abs(mu_t - pv32.mean(axis=0)) <= bound)
