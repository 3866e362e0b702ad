"""The network's CUDA forward/backward/Adam against the FP64 reference that
sees the same bfloat16-rounded operands (oracle.mlp), element by element.

Per-element bound.  Both sides round the same FP32 values to bfloat16 (weights,
inputs, the output gradient), so what remains is (1) the FP32 accumulation of
the tensor-core products (exact in FP32: 8-bit by 8-bit significands) in an
order the oracle does not follow, at most gamma(K) sum_k |a_k b_k| with
gamma(K) = K 2^-23 (twice the (K-1) 2^-24 of any round-to-nearest summation
order, as the tensor core's internal accumulation is not specified), plus
2^-24 |v| for the FP32 bias add; and (2) where that error can carry a value
across a bfloat16 rounding boundary (or across 0 under ReLU), the re-rounded
activation or gradient differs by the resulting jump.  q = bf16(relu(.)) is
monotone, so the largest jump over [v - e, v + e] is at an end of it.  The
bounds below propagate these per-element intervals through the network
exactly as the two sides compute it; nothing is loosened to a norm.
"""
import numpy as np
import pytest

from oracle import mlp as omlp

pytestmark = pytest.mark.gpu

U = 2.0 ** -24


def gamma(K):
    return K * 2.0 ** -23


def q_relu(v):
    return omlp.bf16_round(np.maximum(v, 0.0))


def jump(fn, v, e, ref):
    """max |fn(t) - ref| over t in [v - e, v + e] for a monotone fn."""
    return np.maximum(np.abs(fn(v + e) - ref), np.abs(fn(v - e) - ref))


def forward_bounds(p, x):
    """Oracle forward with per-element bounds on |GPU - oracle| of h1, h2, y."""
    y, c = omlp.forward(p, x, bf16=True)
    xr, W1, W2, W3 = c["x"], np.abs(c["W1"]), np.abs(c["W2"]), np.abs(c["W3"])
    v1 = c["x"] @ c["W1"].T + p["b1"]
    a1 = gamma(xr.shape[1]) * (np.abs(xr) @ W1.T)
    e1 = a1 + U * (np.abs(v1) + a1)
    d1 = jump(q_relu, v1, e1, c["h1"])
    v2 = c["h1"] @ c["W2"].T + p["b2"]
    a2 = d1 @ W2.T + gamma(W2.shape[1]) * ((np.abs(c["h1"]) + d1) @ W2.T)
    e2 = a2 + U * (np.abs(v2) + a2)
    d2 = jump(q_relu, v2, e2, c["h2"])
    a3 = d2 @ W3.T + gamma(W3.shape[1]) * ((np.abs(c["h2"]) + d2) @ W3.T)
    ey = a3 + U * (np.abs(y) + a3)
    return y, c, {"v1": v1, "v2": v2, "e2": e2, "d1": d1, "d2": d2, "ey": ey}


def grad_bounds(p, x, t):
    """Oracle loss and gradients with per-element bounds on |GPU - oracle|."""
    rl, rg = omlp.loss_and_grads(p, x, t, bf16=True)
    y, c, f = forward_bounds(p, x)
    B, n_out = y.shape
    s = 1.0 / (B * n_out)
    s32 = float(np.float32(s))                       # the kernel's FP32 scale
    sb = omlp.bf16_round(np.array([s]))[0]
    ds = abs(omlp.bf16_round(np.array([s32]))[0] - sb)
    diff = y - t
    flip = np.abs(diff) <= f["ey"]                   # the sign of y - t may differ
    dyr = omlp.bf16_round(np.sign(diff) * s)
    Ddy = np.where(flip, 2 * sb, 0.0) + ds
    W2, W3 = np.abs(c["W2"]), np.abs(c["W3"])
    h1, h2, d1, d2 = c["h1"], c["h2"], f["d1"], f["d2"]
    bd = {}
    bd["W3"] = Ddy.T @ (h2 + d2) + np.abs(dyr).T @ d2 + gamma(B) * (
        (np.abs(dyr) + Ddy).T @ (h2 + d2))
    bd["b3"] = np.where(flip, 2 * s32, 0.0).sum(axis=0) + B * abs(s32 - s) + gamma(B) * B * s32

    def masked_back(dr, Dd, W, h, dh, v, e):
        g = dr @ W
        eg = Dd @ np.abs(W) + gamma(W.shape[0]) * ((np.abs(dr) + Dd) @ np.abs(W))
        # the ReLU mask comes from the GPU's own activation, which may sit on the
        # other side of 0 where the interval around the oracle's value reaches it
        mflip = (dh > 0) & ((h == 0) | (q_relu(v - e) == 0))
        dv = g * (h > 0)
        Dv = np.where(mflip, np.abs(g) + eg, np.where(h > 0, eg, 0.0))
        vr = omlp.bf16_round(dv)
        Dvr = jump(lambda z: omlp.bf16_round(z), dv, Dv, vr)
        return dv, Dv, vr, Dvr

    e1 = None  # the layer-1 interval half-width, recomputed for its mask
    xr = c["x"]
    a1 = gamma(xr.shape[1]) * (np.abs(xr) @ np.abs(c["W1"]).T)
    e1 = a1 + U * (np.abs(f["v1"]) + a1)
    dh2, Ddh2, dh2r, Ddh2r = masked_back(dyr, Ddy, c["W3"], h2, d2, f["v2"], f["e2"])
    bd["W2"] = Ddh2r.T @ (h1 + d1) + np.abs(dh2r).T @ d1 + gamma(B) * (
        (np.abs(dh2r) + Ddh2r).T @ (h1 + d1))
    bd["b2"] = Ddh2.sum(axis=0) + gamma(B) * (np.abs(dh2) + Ddh2).sum(axis=0)
    dh1, Ddh1, dh1r, Ddh1r = masked_back(dh2r, Ddh2r, c["W2"], h1, d1, f["v1"], e1)
    bd["W1"] = Ddh1r.T @ np.abs(xr) + gamma(B) * ((np.abs(dh1r) + Ddh1r).T @ np.abs(xr))
    bd["b1"] = Ddh1.sum(axis=0) + gamma(B) * (np.abs(dh1) + Ddh1).sum(axis=0)
    lbound = s * (f["ey"].sum() + gamma(B * n_out) * np.abs(diff).sum()) + 1e-7 * rl
    return rl, rg, bd, lbound


@pytest.fixture(scope="module")
def ctx():
    from paper_1308_5467_gb300 import dos
    c = dos.Context(0)
    yield c
    c.close()


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
    ref, _, f = forward_bounds(p, x.astype(np.float64))
    err = np.abs(y - ref)
    print("forward: max |dy| %.2e, max |dy| / bound %.3f" % (err.max(), (err / f["ey"]).max()))
    assert np.all(err <= f["ey"])
    assert np.array_equal(net.dos_mlp_get_params(), omlp.flatten(p).astype(np.float32))


@pytest.mark.parametrize("dims,B", [((64, 512, 256), 256), ((13, 40, 7), 5), ((100, 96, 130), 67)])
def test_gradient_parity(ctx, dims, B):
    net, p = make(ctx, *dims, seed=7 + B)
    rng = np.random.default_rng(2)
    x = rng.uniform(-1, 1, (B, dims[0])).astype(np.float32)
    t = rng.uniform(-1, 1, (B, dims[2])).astype(np.float32)
    loss, g = net.dos_mlp_loss_grad(x, t)
    rloss, rg, bd, lbound = grad_bounds(p, x.astype(np.float64), t.astype(np.float64))
    assert abs(loss - rloss) <= lbound
    gg = omlp.unflatten(g, *dims)
    for k in omlp.PARAM_ORDER:
        err = np.abs(gg[k] - rg[k])
        print(k, "max |dg| %.2e, max |dg| / bound %.3f" % (err.max(), (err / np.maximum(
            bd[k], 1e-300)).max()))
        assert np.all(err <= bd[k]), k


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


def test_infer_any_batch_equals_forward(ctx):
    """dos_mlp_infer slices any number of rows through bounded buffers; every row
    equals dos_mlp_forward's bit for bit (rows do not interact in the network)."""
    net, p = make(ctx, 64, 512, 256, seed=21)
    rng = np.random.default_rng(6)
    x = rng.uniform(-1, 1, (70001, 64)).astype(np.float32)  # beyond one forward batch
    y = net.dos_mlp_infer(x, max_rows=4096)
    for a, b in ((0, 3000), (4090, 4100), (65530, 65536), (69000, 70001)):
        assert np.array_equal(y[a:b], net.dos_mlp_forward(x[a:b]))
    import torch
    xd = torch.from_numpy(x[:5000]).cuda()
    yd = torch.empty((5000, 256), dtype=torch.float32, device="cuda")
    net.dos_mlp_infer(xd, out=yd)
    torch.cuda.synchronize()
    assert np.array_equal(yd.cpu().numpy(), y[:5000])
    # FP64 rows of moments read in place (mu_1..mu_64 of rows of 65), host and device
    mu = np.concatenate([np.ones((3000, 1)), rng.uniform(-1, 1, (3000, 64))], axis=1)
    want = net.dos_mlp_forward(mu[:, 1:].astype(np.float32))
    assert np.array_equal(net.dos_mlp_infer(mu, col0=1, max_rows=1000), want)
    assert np.array_equal(net.dos_mlp_infer(torch.from_numpy(mu).cuda(), col0=1), want)


def test_save_load_round_trip_is_bitwise(ctx, tmp_path):
    """A checkpoint restores parameters, Adam moments and the step count: the loaded
    network infers and keeps training bit for bit like the saved one, and the file's
    bytes depend only on the network state."""
    from paper_1308_5467_gb300 import dos
    rng = np.random.default_rng(8)
    X = rng.uniform(-1, 1, (256, 64)).astype(np.float32)
    T = rng.uniform(-1, 1, (256, 256)).astype(np.float32)
    net = dos.MLP(ctx, 64, 512, 256, seed=4)
    for i in range(5):
        net.dos_mlp_train_step(X[i * 32:(i + 1) * 32], T[i * 32:(i + 1) * 32], 1e-3)
    f1, f2, f3 = (str(tmp_path / n) for n in ("a.dosmlp", "b.dosmlp", "c.dosmlp"))
    net.dos_mlp_save(f1)
    net.dos_mlp_save(f2)
    loaded = dos.MLP.dos_mlp_load(ctx, f1)
    loaded.dos_mlp_save(f3)
    raw = open(f1, "rb").read()
    assert raw == open(f2, "rb").read() == open(f3, "rb").read()
    assert raw[:8] == b"DOSMLP\x00\x01" and len(raw) == 8 + 16 + 16 + 12 * net.n_params + 8
    assert (loaded.n_in, loaded.n_hidden, loaded.n_out) == (64, 512, 256)
    assert np.array_equal(loaded.dos_mlp_get_params(), net.dos_mlp_get_params())
    assert np.array_equal(loaded.dos_mlp_infer(X), net.dos_mlp_infer(X))
    for i in range(5, 8):   # Adam state and step count restored: training continues alike
        la = net.dos_mlp_train_step(X[i * 32:(i + 1) * 32], T[i * 32:(i + 1) * 32], 1e-3)
        lb = loaded.dos_mlp_train_step(X[i * 32:(i + 1) * 32], T[i * 32:(i + 1) * 32], 1e-3)
        assert la == lb
    assert np.array_equal(loaded.dos_mlp_get_params(), net.dos_mlp_get_params())


def test_load_rejects_damaged_files(ctx, tmp_path):
    from paper_1308_5467_gb300 import dos
    net = dos.MLP(ctx, 8, 16, 4, seed=1)
    good = str(tmp_path / "good.dosmlp")
    net.dos_mlp_save(good)
    raw = bytearray(open(good, "rb").read())
    cases = {"missing": None, "magic": b"DOSMLX" + bytes(raw[6:]),
             "truncated": bytes(raw[:-9]), "flipped": bytes(raw[:40]) + bytes([raw[40] ^ 1])
             + bytes(raw[41:])}
    for name, content in cases.items():
        path = str(tmp_path / (name + ".dosmlp"))
        if content is not None:
            open(path, "wb").write(content)
        with pytest.raises(dos.DosError) as ei:
            dos.MLP.dos_mlp_load(ctx, path)
        assert ei.value.status == dos.DOS_EIO, name
    assert dos.MLP.dos_mlp_load(ctx, good).n_params == net.n_params
