"""The learned part end to end at a reduced, stated size (the benchmark's
--workload learned runs the configured 20,000 instances with n from 4,096 to
64,000): 960 generated instances (two thirds Anderson lattices, one third
Chung-Lu graphs, n from 4,096 to 16,000), 96 of them held out; moments from 4
start vectors -> network -> DOS, trained by the library's kernels on data the
library generates, scored in the paper's smoothed L1 metric against the
n_v = 1024, M = 256 reference, and compared with plain Jackson KPM from the
same 4 vectors."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

COUNT, HELD, N_LO, N_HI, SEED = 960, 96, 4096, 16000, 11


@pytest.fixture(scope="module")
def ctx():
    from paper_1308_5467_gb300 import dos
    c = dos.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def data(ctx):
    from paper_1308_5467_gb300 import learned
    from synthetic.instances import learned_instance_specs, stream_instances
    specs = learned_instance_specs(COUNT, SEED, N_LO, N_HI)
    stream = stream_instances(specs, window=128)
    test = learned.make_dataset(ctx, (next(stream) for _ in range(HELD)), SEED, b0=0,
                                keep_groups=True)
    train = learned.make_dataset(ctx, stream, SEED, b0=HELD)
    return train, test


def test_grid_moments_roundtrip(ctx):
    # DCT pair: reconstructing undamped moments on N Chebyshev nodes and taking
    # moments back returns them for k < N.
    rng = np.random.default_rng(0)
    mu = np.concatenate([[1.0], rng.uniform(-0.2, 0.2, 99)])
    phi = ctx.dos_reconstruct(mu, 99, "none", N_t=256)
    back = ctx.dos_moments_from_grid(phi, 99)
    assert np.abs(back - mu).max() < 1e-12


def test_dataset_shapes_and_bounds(data):
    train, test = data
    assert train["x"].shape == (COUNT - HELD, 64) and train["y"].shape == (COUNT - HELD, 256)
    assert test["x"].shape == (HELD, 64) and test["mu_ref"].shape == (HELD, 257)
    assert np.all(train["n"] >= N_LO) and np.all(train["n"] <= N_HI)
    lap = np.concatenate([train["laplacian"], test["laplacian"]])
    assert 0.2 < lap.mean() < 0.45        # about one Chung-Lu graph per two lattices
    # normalized Laplacians get [0, 2] padded; every moment stays within mu_0
    assert np.all(test["lb"][test["laplacian"]] == -0.02)
    assert np.all(np.abs(train["mu_in"]) <= 1.0 + 1e-6)


def test_network_beats_jackson_kpm_at_four_vectors(ctx, data):
    from paper_1308_5467_gb300 import learned
    train, test = data
    net = learned.train(ctx, train["x"], train["y"], steps=3000, batch=128, lr=1e-3, seed=3)
    e_kpm, e_net = learned.score(ctx, test, net)
    print("held-out smoothed L1: Jackson KPM (n_v=4) %.4f, network %.4f"
          % (e_kpm.mean(), e_net.mean()))
    assert np.all(np.isfinite(e_net))
    assert e_net.mean() < 0.5 * e_kpm.mean()
    # the serving pipeline (bounds, sweep, network reading the moments in place)
    # gives the network's output on the dataset's inputs bit for bit
    pipe = learned.LearnedPipeline(ctx, net, test["groups"], SEED)
    out = pipe.run().cpu().numpy()
    assert np.array_equal(out, net.dos_mlp_infer(test["x"]))
    # plain KPM with more vectors approaches the reference (the stochastic part shrinks)
    e4 = learned.kpm_errors(ctx, test, 4, 256, SEED)
    e64 = learned.kpm_errors(ctx, test, 64, 256, SEED)
    assert e64.mean() < e4.mean()
