"""Pins of the learned-direction oracle (network, loss, optimiser) against
library routines, adjoint identities and finite differences."""
import numpy as np
import pytest
import scipy.signal

from oracle import learned as L


def _rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def test_conv_matches_scipy_correlate():
    x = _rand((2, 9, 11), 0)
    W = _rand((3, 2, 3, 3), 1)
    got = L.conv(x, W)
    want = np.zeros((3, 9, 11))
    for co in range(3):
        for ci in range(2):
            want[co] += scipy.signal.correlate2d(x[ci], W[co, ci], mode="same", boundary="fill")
    assert np.allclose(got, want, atol=1e-12)


def test_conv_transpose_is_adjoint():
    x = _rand((4, 7, 8), 2)
    W = _rand((5, 4, 3, 3), 3)
    d = _rand((5, 7, 8), 4)
    assert np.isclose(np.sum(L.conv(x, W) * d), np.sum(x * L.conv_transpose(d, W)), rtol=1e-12)


def test_conv_wgrad_is_the_linear_derivative():
    x = _rand((3, 6, 6), 5)
    W = _rand((2, 3, 3, 3), 6)
    dW = _rand((2, 3, 3, 3), 7)
    d = _rand((2, 6, 6), 8)
    lhs = np.sum((L.conv(x, W + dW) - L.conv(x, W)) * d)
    assert np.isclose(lhs, np.sum(dW * L.conv_wgrad(d, x)), rtol=1e-10)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    v = np.concatenate([_rand(2000, 9).astype(np.float32),
                        np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -9, -2.5, 0.0, 1e-30, 3e38], dtype=np.float32)])
    want = torch.from_numpy(v).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(L.bf16(v), want)
    assert L.bf16(np.float32(1 + 2 ** -8)) == 1.0            # tie to even
    assert L.bf16(np.float32(1 + 3 * 2 ** -9)) == np.float32(1 + 2 ** -7)


def test_network_backward_matches_finite_differences():
    """FP64 network (no bf16 rounding): analytic gradient of the angle loss
    against central differences along random parameter directions."""
    n1 = 7
    rng = np.random.default_rng(11)
    theta = L.init_params(3).astype(np.float64)
    rhat = rng.standard_normal((n1, n1))
    c = rng.standard_normal((n1, n1)) * 0.3
    e = rng.standard_normal(n1 * n1)
    M = rng.standard_normal((n1 * n1, n1 * n1))
    A = M @ M.T + n1 * n1 * np.eye(n1 * n1)              # SPD stand-in for the operator

    def loss(th):
        y, _ = L.forward(th, rhat, c, emulate=False)
        y = y.reshape(-1)
        return L.angle_loss(y, e, A @ y, A @ e)[0]

    y, cache = L.forward(theta, rhat, c, emulate=False)
    y = y.reshape(-1)
    _, dy = L.angle_loss(y, e, A @ y, A @ e)
    g = L.backward(cache, dy.reshape(n1, n1))
    for k in range(4):
        d = rng.standard_normal(theta.size)
        h = 1e-6
        fd = (loss(theta + h * d) - loss(theta - h * d)) / (2 * h)
        assert np.isclose(fd, g @ d, rtol=1e-5, atol=1e-9), (fd, g @ d)


def test_angle_loss_invariances_and_gradient():
    rng = np.random.default_rng(12)
    n = 30
    M = rng.standard_normal((n, n))
    A = M @ M.T + n * np.eye(n)
    e = rng.standard_normal(n)
    y = rng.standard_normal(n)
    L1, g = L.angle_loss(y, e, A @ y, A @ e)
    L2, _ = L.angle_loss(3.7 * y, e, A @ (3.7 * y), A @ e)
    assert np.isclose(L1, L2)                                  # scale invariant
    assert np.isclose(L.angle_loss(-2 * e, e, A @ (-2 * e), A @ e)[0], 0.0, atol=1e-14)
    assert 0.0 <= L1 <= 1.0
    d = rng.standard_normal(n)
    h = 1e-6
    fd = (L.angle_loss(y + h * d, e, A @ (y + h * d), A @ e)[0] - L.angle_loss(y - h * d, e, A @ (y - h * d), A @ e)[0]) / (2 * h)
    assert np.isclose(fd, g @ d, rtol=1e-6, atol=1e-10)


def test_adam_first_step_is_lr_times_sign():
    theta = np.array([1.0, -2.0, 0.5])
    g = np.array([3.0, -0.01, 0.0])
    th, m, v = L.adam_step(theta, g, np.zeros(3), np.zeros(3), 1, lr=0.1, eps=1e-12)
    assert np.allclose(th, theta - 0.1 * np.sign(g), atol=1e-9)


def test_param_count_and_packing():
    th = L.init_params(1)
    assert th.size == L.n_params() == 16 * 2 * 9 + 2 * 16 * 16 * 9 + 16 * 9
    assert np.array_equal(L.pack(L.unpack(th)), th)
    b = np.sqrt(6.0 / (2 * 9))
    assert np.abs(L.unpack(th)[0]).max() <= b


# -- the 3D vector network of the elasticity problem (3x3x3 convolutions)

def test_conv3_matches_scipy_correlate():
    x = _rand((2, 5, 6, 7), 20)
    W = _rand((3, 2, 3, 3, 3), 21)
    got = L.conv3(x, W)
    want = np.zeros((3, 5, 6, 7))
    for co in range(3):
        for ci in range(2):
            want[co] += scipy.signal.correlate(x[ci], W[co, ci], mode="same")
    assert np.allclose(got, want, atol=1e-12)


def test_conv3_transpose_is_adjoint():
    x = _rand((4, 5, 4, 6), 22)
    W = _rand((3, 4, 3, 3, 3), 23)
    d = _rand((3, 5, 4, 6), 24)
    assert np.isclose(np.sum(L.conv3(x, W) * d), np.sum(x * L.conv3_transpose(d, W)), rtol=1e-12)


def test_conv3_wgrad_is_the_linear_derivative():
    x = _rand((3, 4, 5, 4), 25)
    W = _rand((2, 3, 3, 3, 3), 26)
    dW = _rand((2, 3, 3, 3, 3), 27)
    d = _rand((2, 4, 5, 4), 28)
    lhs = np.sum((L.conv3(x, W + dW) - L.conv3(x, W)) * d)
    assert np.isclose(lhs, np.sum(dW * L.conv3_wgrad(d, x)), rtol=1e-10)


def test_image3_layout_is_component_fastest():
    Z, Y, X = 2, 3, 4
    v = np.arange(3 * Z * Y * X, dtype=float)
    img = L.to_image3(v, (Z, Y, X))
    # unknown i = a + 3 * (x + X (y + Y z))
    for a, z, y, x in ((0, 0, 0, 0), (2, 1, 2, 3), (1, 0, 1, 2)):
        assert img[a, z, y, x] == a + 3 * (x + X * (y + Y * z))
    assert np.array_equal(L.from_image3(img), v)


def test_network3_backward_matches_finite_differences():
    """FP64 3D network: analytic gradient of the angle loss against central
    differences along random parameter directions."""
    shape = (3, 4, 3)
    n = 3 * 3 * 4 * 3
    rng = np.random.default_rng(13)
    theta = L.init_params3(3).astype(np.float64)
    assert theta.size == L.n_params3() == 16416
    rhat = rng.standard_normal(n)
    e = rng.standard_normal(n)
    Mx = rng.standard_normal((n, n))
    A = Mx @ Mx.T + n * np.eye(n)

    def loss(th):
        y, _ = L.forward3(th, L.to_image3(rhat, shape), emulate=False)
        y = L.from_image3(y)
        return L.angle_loss(y, e, A @ y, A @ e)[0]

    _, g = L.batch_grad3(theta, [(rhat, e, A)], shape, emulate=False)
    for k in range(3):
        d = rng.standard_normal(theta.size)
        h = 1e-6
        fd = (loss(theta + h * d) - loss(theta - h * d)) / (2 * h)
        assert np.isclose(fd, g @ d, rtol=1e-5, atol=1e-9), (fd, g @ d)


def test_network3_planted_tap_swap_is_seen():
    """A weight applied at the mirrored tap (the mistake an adjoint written
    with the wrong flip makes) changes the forward output."""
    shape = (4, 4, 4)
    rng = np.random.default_rng(14)
    theta = L.init_params3(5).astype(np.float64)
    rhat = L.to_image3(rng.standard_normal(3 * 64), shape)
    y0, _ = L.forward3(theta, rhat, emulate=False)
    Ws = L.unpack3(theta.copy())
    Ws[1] = Ws[1][:, :, ::-1, :, :].copy()
    y1, _ = L.forward3(np.concatenate([W.reshape(-1) for W in Ws]), rhat, emulate=False)
    assert np.abs(y1 - y0).max() > 1e-3 * np.abs(y0).max()
