"""Pins of the learned-initialiser oracle (oracle/unet.py) to things other than itself:
the direct-sum definition of the convolution, scipy's 2D correlation, adjointness of
every linear layer, central-difference gradients of the whole network, and torch's
float32 -> bfloat16 conversion. CPU only."""
import numpy as np
import pytest

from oracle import unet as U

rng = np.random.default_rng(1234)


def test_conv_matches_the_direct_sum():
    x = rng.normal(size=(2, 5, 6, 3))
    w = rng.normal(size=(4, 9, 3))
    assert np.allclose(U.conv3x3(x, w), U.conv3x3_direct(x, w), atol=1e-12)


def test_conv_matches_scipy_correlation():
    signal = pytest.importorskip("scipy.signal")
    x = rng.normal(size=(1, 7, 9, 2))
    w = rng.normal(size=(3, 9, 2))
    out = U.conv3x3(x, w)
    for co in range(3):
        ref = np.zeros((7, 9))
        for ci in range(2):
            k = w[co, :, ci].reshape(3, 3)  # [dy + 1, dx + 1]: a correlation kernel
            ref += signal.correlate2d(x[0, :, :, ci], k, mode="same", boundary="fill", fillvalue=0.0)
        assert np.allclose(out[0, :, :, co], ref, atol=1e-12)


def test_linear_layers_are_adjoint_pairs():
    x = rng.normal(size=(2, 8, 6, 3))
    w = rng.normal(size=(5, 9, 3))
    y = rng.normal(size=(2, 8, 6, 5))
    assert np.isclose(np.sum(U.conv3x3(x, w) * y), np.sum(x * U.conv3x3_grad_input(y, w)), rtol=1e-12)
    # weight gradient: d <conv(x, w), y> / dw
    gw = U.conv3x3_grad_weight(x, y)
    dw = rng.normal(size=w.shape)
    assert np.isclose(np.sum(U.conv3x3(x, dw) * y), np.sum(gw * dw), rtol=1e-12)
    p = rng.normal(size=(2, 4, 3, 3))
    assert np.isclose(np.sum(U.avgpool2(x) * p), np.sum(x * U.avgpool2_backward(p)), rtol=1e-12)
    q = rng.normal(size=(2, 16, 12, 3))
    assert np.isclose(np.sum(U.upsample2(x) * q), np.sum(x * U.upsample2_backward(q)), rtol=1e-12)


def test_shift_direction():
    x = np.zeros((1, 4, 4, 1))
    x[0, 2, 1, 0] = 1.0
    s = U.shift(x, 1, -1)  # s[y, x] = x[y + 1, x - 1]
    assert s[0, 1, 2, 0] == 1.0 and s.sum() == 1.0


def test_network_gradient_against_central_differences():
    widths = (2, 3, 4, 5)
    cin, C, S, N = 3, 2, 16, 2
    n = U.num_params(widths, cin, U.COUT)
    theta = rng.normal(size=n) * 0.3
    x = rng.normal(size=(N, S, S, cin))
    target = rng.normal(size=(N, C, S, S)) * 0.1

    def loss(th):
        out, _ = U.forward(th, x, widths, bf16=False)
        return U.mse(out, target, C)[0]

    out, cache = U.forward(theta, x, widths, bf16=False)
    _, gout = U.mse(out, target, C)
    g = U.backward(theta, cache, gout, widths, bf16=False)
    idx = rng.choice(n, size=40, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros(n)
        e[i] = h
        fd = (loss(theta + e) - loss(theta - e)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-8, (i, fd, g[i])


def test_parameter_count_of_the_library_network():
    assert U.num_params() == 304720


def test_bf16_rounding_ties_to_even_and_matches_torch():
    one = 1.0
    assert U.round_bf16(one) == 1.0
    assert U.round_bf16(1.0 + 2.0 ** -8) == 1.0                        # tie -> even (down)
    assert U.round_bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6        # tie -> even (up)
    assert U.round_bf16(1.0 + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7
    torch = pytest.importorskip("torch")
    v = rng.normal(size=10000) * np.exp(rng.uniform(-20, 20, size=10000))
    ref = torch.tensor(v, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(U.round_bf16(v), ref)


def test_adam_first_update_is_the_normalised_gradient():
    """Bias correction makes update 1 exactly -lr g / (|g| + eps): m_hat = g and
    v_hat = g^2 after one step from zero moments."""
    g = np.array([3.0, -0.5, 1e-9, -2e-8, 0.0, 7e4])
    theta = rng.normal(size=g.size)
    lr, eps = 1e-3, 1e-8
    t1, m1, v1 = U.adam_step(theta, np.zeros_like(g), np.zeros_like(g), g, 1, lr)
    assert np.allclose(t1, theta - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    assert np.allclose(m1, 0.1 * g, rtol=1e-15) and np.allclose(v1, 0.001 * g * g, rtol=1e-15)


def test_adam_constant_gradient_keeps_the_step_size():
    """With a constant gradient the corrected moments stay g and g^2 at every update
    (sum_k (1 - b) b^k over t terms = 1 - b^t), so each step is lr g / (|g| + eps)."""
    g = np.array([0.25, -4.0])
    theta, m, v = np.zeros(2), np.zeros(2), np.zeros(2)
    for t in range(1, 8):
        theta, m, v = U.adam_step(theta, m, v, g, t, 0.01)
    assert np.allclose(theta, -7 * 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_adam_two_updates_worked_by_hand():
    """g = +1 then -1: m_2 = 0.9 * 0.1 - 0.1 = -0.01, m_hat = -0.01 / 0.19 = -1/19;
    v_2 = 0.999 * 0.001 + 0.001 = 0.001999 = 1 - 0.999^2, v_hat = 1. So
    theta_2 = theta_0 - lr / (1 + eps) + lr / (19 (1 + eps)).
    g = +1 then 0: m_hat = 0.09 / 0.19 = 9/19, v_hat = 0.000999 / 0.001999 = 999/1999."""
    lr, eps = 0.05, 1e-8
    th, m, v = U.adam_step(np.zeros(2), np.zeros(2), np.zeros(2), np.array([1.0, 1.0]), 1, lr)
    th, m, v = U.adam_step(th, m, v, np.array([-1.0, 0.0]), 2, lr)
    assert th[0] == pytest.approx(-lr / (1 + eps) + lr / (19 * (1 + eps)), rel=1e-13)
    assert th[1] == pytest.approx(-lr / (1 + eps) - lr * (9 / 19) / (np.sqrt(999 / 1999) + eps), rel=1e-13)
    assert m[0] == pytest.approx(-0.01, rel=1e-13) and v[0] == pytest.approx(0.001999, rel=1e-13)
