"""The heat-capacity observable (Section 4.3) on the GPU against the oracle,
from KPM moments and from Lanczos Ritz pairs, and the paper's comparison of the
two at M = 40 in the error of Eq. errormetric_g."""
import numpy as np
import pytest

from oracle import observables as obs
from synthetic import laplacian_2d

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1308_5467_gb300 import dos
    c = dos.Context(0)
    yield c
    c.close()


def test_heat_capacity_kpm_and_points_parity(ctx):
    from paper_1308_5467_gb300 import dos
    A = laplacian_2d(30)
    lam = np.linalg.eigvalsh(A.to_dense())
    lb, ub = -0.08, 8.08
    betas = np.geomspace(0.05, 20.0, 25)
    Ad = dos.CSRArrays.from_synthetic(A, device="cuda")
    mu = ctx.dos_kpm_moments(Ad, lb, ub, 40, 100, seed=1, precision="f64")
    got = ctx.dos_heat_capacity(betas, mu=mu, lb=lb, ub=ub)
    ref = obs.heat_capacity_kpm(mu, "jackson", lb, ub, betas)
    assert np.abs(got - ref).max() < 1e-11
    exact = ctx.dos_heat_capacity(betas, pts=lam, wts=np.ones_like(lam))
    assert np.abs(exact - obs.heat_capacity_points(lam, np.ones_like(lam), betas)).max() < 1e-12
    theta, weight, _ = ctx.dos_lanczos_ritz(Ad, 40, 100, seed=1)
    lan = ctx.dos_heat_capacity(betas, pts=theta, wts=weight)
    assert np.abs(lan - obs.heat_capacity_points(theta, weight, betas)).max() < 1e-12
    # Eq. errormetric_g for both methods, C_v normalised to a maximum of one (Section 4.3)
    e_kpm = np.abs(got / exact.max() - exact / exact.max()).max()
    e_lan = np.abs(lan / exact.max() - exact / exact.max()).max()
    print("heat capacity, M = 40, n_v = 100: max error KPM %.2e, Lanczos %.2e" % (e_kpm, e_lan))
    assert e_kpm < 0.05 and e_lan < 0.05
