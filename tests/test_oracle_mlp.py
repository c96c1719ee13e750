"""Pins of the FP64 MLP oracle: its gradient against central finite
differences of its own loss, Adam's first step against its closed form, and
bfloat16 rounding against hand-checked bit patterns."""
import numpy as np
import pytest

from oracle import mlp


def _params(rng, scale=0.5):
    return rng.normal(scale=scale, size=mlp.N_PARAMS)


def test_parameter_count_matches_library():
    assert mlp.N_PARAMS == 16 * 64 + 64 + 64 * 64 + 64 + 64 + 1 == 5313


@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_matches_central_differences(seed):
    rng = np.random.default_rng(seed)
    theta = _params(rng)
    X = rng.normal(size=(23, 16))
    t = rng.normal(size=23)
    _, g = mlp.loss_grad(theta, X, t)
    idx = rng.choice(mlp.N_PARAMS, 60, replace=False)
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss_grad(tp, X, t)[0] - mlp.loss_grad(tm, X, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_adam_first_step_is_sign_times_lr():
    rng = np.random.default_rng(2)
    theta = _params(rng)
    grad = rng.normal(size=mlp.N_PARAMS)
    z = np.zeros_like(theta)
    new, m, v = mlp.adam_step(theta, grad, z, z, 1, lr=1e-3, eps=0.0)
    np.testing.assert_allclose(new - theta, -1e-3 * np.sign(grad), rtol=1e-12, atol=0)
    np.testing.assert_allclose(m, 0.1 * grad, rtol=1e-15)
    np.testing.assert_allclose(v, 0.001 * grad * grad, rtol=1e-12)


def test_bf16_rounding_bit_patterns():
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties to even -> 1
    assert mlp.bf16(np.float32(1.0 + 2 ** -8)) == 1.0
    # 1 + 3 * 2^-8 is halfway between 1 + 2^-7 and 1 + 2^-6: ties to even -> 1 + 2^-6
    assert mlp.bf16(np.float32(1.0 + 3 * 2 ** -8)) == 1.0 + 2 ** -6
    # just above a tie rounds up
    assert mlp.bf16(np.float32(1.0 + 2 ** -8 + 2 ** -20)) == 1.0 + 2 ** -7
    # values with 8 significant bits are kept
    for v in (0.5, -3.0, 1.0 + 2 ** -7, 2.0 ** -100):
        assert mlp.bf16(np.float32(v)) == v
