"""Pins of the FP64 network reference: the backward pass against central finite
differences, the forward pass against explicit per-sample loops, the bfloat16
rounding against exactly representable values and ties, and one Adam step
against its closed form for a scalar."""
import numpy as np
import pytest

from oracle import mlp


def test_bf16_round_exact_and_ties():
    exact = np.array([0.0, 1.0, -2.0, 0.15625, 3.0 * 2.0 ** -100])
    assert np.array_equal(mlp.bf16_round(exact), exact)
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties to even -> 1
    assert mlp.bf16_round(np.array([1.0 + 2.0 ** -8]))[0] == 1.0
    # 1 + 3*2^-8 is halfway between 1 + 2^-7 and 1 + 2^-6: ties to even -> 1 + 2^-6
    assert mlp.bf16_round(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6
    assert mlp.bf16_round(np.array([1.0 + 2.0 ** -8 + 2.0 ** -20]))[0] == 1.0 + 2.0 ** -7
    r = np.random.default_rng(0).standard_normal(1000)
    assert np.all(np.abs(mlp.bf16_round(r) - r) <= np.abs(r) * 2.0 ** -8)


def test_forward_matches_per_sample_loops():
    p = mlp.init_params(5, 7, 3, seed=1)
    p["b1"] = np.linspace(-0.2, 0.3, 7)
    p["b2"] = np.linspace(0.1, -0.1, 7)
    p["b3"] = np.array([0.5, -0.5, 0.0])
    x = np.random.default_rng(2).standard_normal((4, 5))
    y, _ = mlp.forward(p, x)
    for b in range(4):
        h1 = [max(0.0, sum(p["W1"][i, k] * x[b, k] for k in range(5)) + p["b1"][i]) for i in range(7)]
        h2 = [max(0.0, sum(p["W2"][i, k] * h1[k] for k in range(7)) + p["b2"][i]) for i in range(7)]
        out = [sum(p["W3"][i, k] * h2[k] for k in range(7)) + p["b3"][i] for i in range(3)]
        assert np.allclose(y[b], out, rtol=0, atol=1e-13)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(3)
    n_in, n_h, n_out, B = 6, 9, 4, 5
    p = mlp.init_params(n_in, n_h, n_out, seed=4)
    p["b1"] = rng.uniform(0.05, 0.2, n_h)   # keep units active, away from kinks
    p["b2"] = rng.uniform(0.05, 0.2, n_h)
    x = rng.standard_normal((B, n_in))
    target = rng.standard_normal((B, n_out)) * 3.0  # away from y: no L1 kink
    loss, g = mlp.loss_and_grads(p, x, target)
    flat = mlp.flatten(p)
    gflat = mlp.flatten(g)
    eps = 1e-6
    for idx in rng.choice(flat.size, size=60, replace=False):
        fp, fm = flat.copy(), flat.copy()
        fp[idx] += eps
        fm[idx] -= eps
        lp, _ = mlp.loss_and_grads(mlp.unflatten(fp, n_in, n_h, n_out), x, target)
        lm, _ = mlp.loss_and_grads(mlp.unflatten(fm, n_in, n_h, n_out), x, target)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - gflat[idx]) <= 1e-7 + 1e-5 * abs(fd), idx


def test_adam_scalar_closed_form():
    # After one step with zero initial moments the bias-corrected update is
    # lr * g / (|g| + eps): a signed step of almost exactly lr.
    p = {"w": np.array([1.0])}
    m = {"w": np.zeros(1)}
    v = {"w": np.zeros(1)}
    p, m, v = mlp.adam_step(p, {"w": np.array([0.25])}, m, v, 1, lr=0.01)
    assert abs(p["w"][0] - (1.0 - 0.01 * 0.25 / (0.25 + 1e-8))) < 1e-15
    p, m, v = mlp.adam_step(p, {"w": np.array([-0.5])}, m, v, 2, lr=0.01)
    m2 = 0.9 * 0.1 * 0.25 + 0.1 * -0.5
    v2 = 0.999 * 0.001 * 0.0625 + 0.001 * 0.25
    expect = (1.0 - 0.01 * 0.25 / (0.25 + 1e-8)) - 0.01 * (m2 / (1 - 0.81)) / (
        np.sqrt(v2 / (1 - 0.999 ** 2)) + 1e-8)
    assert abs(p["w"][0] - expect) < 1e-15


def test_param_count_of_the_configured_network():
    p = mlp.init_params(64, 512, 256, seed=0)
    assert mlp.flatten(p).size == 427264
