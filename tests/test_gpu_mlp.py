"""The network's CUDA forward/backward/Adam against the FP64 reference that
sees the same bfloat16-rounded operands (oracle.mlp)."""
import numpy as np
import pytest

from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1308_5467_gb300 import dos
    c = dos.Context(0)
    yield c
    c.close()


def rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30)


def make(ctx, n_in, n_h, n_out, seed):
    from paper_1308_5467_gb300 import dos
    net = dos.MLP(ctx, n_in, n_h, n_out, seed=seed)
    p = omlp.init_params(n_in, n_h, n_out, seed)
    rng = np.random.default_rng(seed)
    for k in ("b1", "b2", "b3"):
        p[k] = rng.uniform(-0.1, 0.1, p[k].shape)
    p = {k: v.astype(np.float32).astype(np.float64) for k, v in p.items()}
    net.dos_mlp_set_params(omlp.flatten(p).astype(np.float32))
    return net, p


@pytest.mark.parametrize("dims,B", [((64, 512, 256), 256), ((13, 40, 7), 5), ((64, 512, 256), 1),
                                    ((100, 96, 130), 67)])
def test_forward_parity(ctx, dims, B):
    net, p = make(ctx, *dims, seed=B)
    x = np.random.default_rng(1).uniform(-1, 1, (B, dims[0])).astype(np.float32)
    y = net.dos_mlp_forward(x)
    ref, _ = omlp.forward(p, x.astype(np.float64), bf16=True)
    assert rel(y, ref) < 1e-2
    assert np.array_equal(net.dos_mlp_get_params(), omlp.flatten(p).astype(np.float32))


@pytest.mark.parametrize("dims,B", [((64, 512, 256), 256), ((13, 40, 7), 5), ((100, 96, 130), 67)])
def test_gradient_parity(ctx, dims, B):
    net, p = make(ctx, *dims, seed=7 + B)
    rng = np.random.default_rng(2)
    x = rng.uniform(-1, 1, (B, dims[0])).astype(np.float32)
    t = rng.uniform(-1, 1, (B, dims[2])).astype(np.float32)
    loss, g = net.dos_mlp_loss_grad(x, t)
    rloss, rg = omlp.loss_and_grads(p, x.astype(np.float64), t.astype(np.float64), bf16=True)
    assert abs(loss - rloss) < 1e-4 * max(1.0, rloss)
    gg = omlp.unflatten(g, *dims)
    for k in omlp.PARAM_ORDER:
        assert rel(gg[k], rg[k]) < 1e-2, k


def test_adam_step_parity(ctx):
    dims, B, lr = (32, 64, 16), 24, 1e-3
    net, p = make(ctx, *dims, seed=3)
    rng = np.random.default_rng(4)
    x = rng.uniform(-1, 1, (B, dims[0])).astype(np.float32)
    t = rng.uniform(-1, 1, (B, dims[2])).astype(np.float32)
    _, g_gpu = net.dos_mlp_loss_grad(x, t)
    net.dos_mlp_train_step(x, t, lr)
    got = net.dos_mlp_get_params().astype(np.float64)
    # Adam applied in FP64 to the library's own gradient
    flat = omlp.flatten(p)
    pp = {"w": flat.copy()}
    m = {"w": np.zeros_like(flat)}
    v = {"w": np.zeros_like(flat)}
    pp, _, _ = omlp.adam_step(pp, {"w": g_gpu.astype(np.float64)}, m, v, 1, lr)
    assert np.abs(got - pp["w"]).max() < 1e-6


def test_training_reduces_loss_and_is_deterministic(ctx):
    from paper_1308_5467_gb300 import dos
    rng = np.random.default_rng(5)
    X = rng.uniform(-1, 1, (512, 64)).astype(np.float32)
    Wt = rng.standard_normal((64, 256)).astype(np.float32) / 8
    T = np.tanh(X @ Wt).astype(np.float32)
    losses = []
    for rep in range(2):
        net = dos.MLP(ctx, 64, 512, 256, seed=11)
        ls = [net.dos_mlp_train_step(X[i % 4 * 128:(i % 4 + 1) * 128],
                                     T[i % 4 * 128:(i % 4 + 1) * 128], 1e-3) for i in range(200)]
        losses.append(ls)
        params = net.dos_mlp_get_params()
        if rep == 0:
            first = params
        else:
            assert np.array_equal(first, params)
        net.close()
    assert losses[0] == losses[1]
    assert np.mean(losses[0][-10:]) < 0.5 * np.mean(losses[0][:5])
