"""The learned part end to end: moments from 4 start vectors -> network -> DOS,
trained by the library's kernels on data the library generates, scored in the
paper's smoothed L1 metric against the n_v = 1024, M = 256 reference, and
compared with plain Jackson KPM from the same 4 vectors."""
import numpy as np
import pytest

from synthetic import anderson_3d, chung_lu_normalized_laplacian

pytestmark = pytest.mark.gpu


def instances(count, seed):
    rng = np.random.default_rng(seed)
    mats = []
    for i in range(count):
        if i % 3 == 2:
            mats.append(chung_lu_normalized_laplacian(int(rng.integers(4000, 12000)),
                                                      seed=int(rng.integers(1 << 30))).astype(np.float32))
        else:
            mats.append(anderson_3d(int(rng.integers(16, 24)), float(rng.uniform(1.0, 16.0)),
                                    int(rng.integers(1 << 30))).astype(np.float32))
    return mats


@pytest.fixture(scope="module")
def ctx():
    from paper_1308_5467_gb300 import dos
    c = dos.Context(0)
    yield c
    c.close()


def test_grid_moments_roundtrip(ctx):
    # DCT pair: reconstructing undamped moments on N Chebyshev nodes and taking
    # moments back returns them for k < N.
    rng = np.random.default_rng(0)
    mu = np.concatenate([[1.0], rng.uniform(-0.2, 0.2, 99)])
    phi = ctx.dos_reconstruct(mu, 99, "none", N_t=256)
    back = ctx.dos_moments_from_grid(phi, 99)
    assert np.abs(back - mu).max() < 1e-12


def test_network_beats_jackson_kpm_at_four_vectors(ctx):
    from paper_1308_5467_gb300 import learned
    train_mats = instances(720, seed=1)
    test_mats = instances(96, seed=2)
    tr = learned.make_dataset(ctx, train_mats, seed=10)
    te = learned.make_dataset(ctx, test_mats, seed=20)
    assert tr["x"].shape == (720, 64) and tr["y"].shape == (720, 256)
    net = learned.train(ctx, tr["x"], tr["y"], steps=2500, batch=128, lr=1e-3, seed=3)
    e_kpm, e_net = learned.score(ctx, te, net)
    print("held-out smoothed L1: Jackson KPM (n_v=4) %.4f, network %.4f"
          % (e_kpm.mean(), e_net.mean()))
    assert np.all(np.isfinite(e_net))
    assert e_net.mean() < e_kpm.mean()
