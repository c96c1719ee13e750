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


def _hand_weights():
    """Weights whose network is a function written out below: hidden layer
    1 copies the inputs (unit i = x_i), adds unit 16 = 2 x_0 and unit 17 =
    0.25 - x_15; layer 2 is 0.5 minus layer 1, plus unit 16 of layer 1 into
    its unit 0; the output weighs hidden unit j by (j + 1) / 64, plus 0.125."""
    W1 = np.zeros((64, 16))
    for i in range(16):
        W1[i, i] = 1.0
    W1[16, 0] = 2.0
    W1[17, 15] = -1.0
    b1 = np.zeros(64)
    b1[17] = 0.25
    W2 = -np.eye(64)
    W2[0, 16] = 1.0
    b2 = np.full(64, 0.5)
    W3 = ((np.arange(64) + 1.0) / 64.0)[None, :]
    b3 = np.array([0.125])
    return mlp.pack({"W1": W1, "b1": b1, "W2": W2, "b2": b2, "W3": W3, "b3": b3})


def _hand_forward(x):
    """The same network, one unit at a time (ReLU written as max(., 0))."""
    relu = lambda v: v if v > 0.0 else 0.0
    h1 = [0.0] * 64
    for i in range(16):
        h1[i] = relu(x[i])
    h1[16] = relu(2.0 * x[0])
    h1[17] = relu(0.25 - x[15])
    h2 = [relu(0.5 - h1[j]) for j in range(64)]
    h2[0] = relu(0.5 - h1[0] + h1[16])
    return 0.125 + sum((j + 1) / 64.0 * h2[j] for j in range(64))


def test_forward_against_a_network_written_out_by_hand():
    """Pins the layer order, the ReLUs and the orientation of every weight
    matrix: a dropped ReLU, swapped layers or a transposed W2 change the
    output on these inputs."""
    theta = _hand_weights()
    rng = np.random.default_rng(3)
    X = np.vstack([rng.normal(scale=0.8, size=(40, 16)),
                   np.linspace(-1.0, 1.0, 16)[None, :],      # some inputs above 0.5, some negative
                   np.zeros((1, 16))])
    y, _ = mlp.forward(theta, X)
    want = np.array([_hand_forward(list(x)) for x in X])
    np.testing.assert_allclose(y, want, rtol=1e-14, atol=1e-14)
    # one value by hand: x = 0 gives h1 = (0, .., 0, 0.25 at unit 17), h2 = 0.5
    # everywhere but unit 17 (0.25): 0.125 + 0.5 * sum((j+1)/64) - 0.25 * 18/64
    assert y[-1] == pytest.approx(0.125 + 0.5 * (64 * 65 / 2) / 64 - 0.25 * 18 / 64, abs=1e-14)
    # the mistakes the pin is there to catch
    P = mlp.unpack(theta)
    no_relu = (np.maximum(0.0, (X @ P["W1"].T + P["b1"]) @ P["W2"].T + P["b2"]) @ P["W3"].T + P["b3"])[:, 0]
    assert np.max(np.abs(no_relu - want)) > 1e-3
    tr = mlp.pack({**P, "W2": P["W2"].T})
    assert np.max(np.abs(mlp.forward(tr, X)[0] - want)) > 1e-3
