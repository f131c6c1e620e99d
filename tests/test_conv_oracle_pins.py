"""Pins of the FP64 convolution oracle: adjoint identities, finite
differences, the 1x1x1 case as a matrix product, and the impulse response."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def conv():
    from oracle import conv as c
    c.build()
    return c


def _rand(rng, *shape):
    return rng.standard_normal(shape)


def test_adjoint_of_forward_is_backward_data(conv):
    rng = np.random.default_rng(1)
    x = _rand(rng, 2, 5, 4, 6, 3)
    w = _rand(rng, 4, 3, 3, 3, 3)
    dy = _rand(rng, 2, 5, 4, 6, 4)
    lhs = np.sum(conv.conv3d_fwd(x, w) * dy)
    rhs = np.sum(x * conv.conv3d_bwd_data(dy, w))
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)


def test_backward_weight_is_the_weight_gradient(conv):
    """<fwd(x; v), dy> is linear in the weights: it equals <dw(x, dy), v>."""
    rng = np.random.default_rng(2)
    x = _rand(rng, 1, 4, 5, 3, 2)
    dy = _rand(rng, 1, 4, 5, 3, 3)
    v = _rand(rng, 3, 3, 3, 3, 2)
    dw, db = conv.conv3d_bwd_weight(x, dy, 3)
    assert abs(np.sum(conv.conv3d_fwd(x, v) * dy) - np.sum(dw * v)) < 1e-11 * np.abs(dw).sum()
    assert np.allclose(db, dy.sum(axis=(0, 1, 2, 3)))


def test_finite_differences(conv):
    """Gradient of L = sum(fwd(x) * g) + 0.5 |fwd(x)|^2 by central differences."""
    rng = np.random.default_rng(3)
    x = _rand(rng, 1, 3, 3, 4, 2)
    w = _rand(rng, 2, 3, 3, 3, 2)
    b = _rand(rng, 2)
    g = _rand(rng, 1, 3, 3, 4, 2)

    def loss(x, w, b):
        y = conv.conv3d_fwd(x, w, b)
        return np.sum(y * g) + 0.5 * np.sum(y * y)

    y = conv.conv3d_fwd(x, w, b)
    dy = g + y
    dx = conv.conv3d_bwd_data(dy, w)
    dw, db = conv.conv3d_bwd_weight(x, dy, 3)
    eps = 1e-6
    for arr, grad in ((x, dx), (w, dw), (b, db)):
        flat = arr.reshape(-1)
        for j in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[j]
            flat[j] = old + eps
            lp = loss(x, w, b)
            flat[j] = old - eps
            lm = loss(x, w, b)
            flat[j] = old
            assert abs((lp - lm) / (2 * eps) - grad.reshape(-1)[j]) < 1e-5 * max(1.0, abs(grad.reshape(-1)[j]))


def test_pointwise_kernel_is_a_matrix_product(conv):
    rng = np.random.default_rng(4)
    x = _rand(rng, 2, 3, 4, 5, 6)
    w = _rand(rng, 7, 1, 1, 1, 6)
    b = _rand(rng, 7)
    y = conv.conv3d_fwd(x, w, b)
    assert np.allclose(y, x @ w[:, 0, 0, 0, :].T + b, atol=1e-12)


def test_impulse_response_is_the_reversed_kernel(conv):
    rng = np.random.default_rng(5)
    w = _rand(rng, 2, 3, 3, 3, 1)
    x = np.zeros((1, 7, 7, 7, 1))
    x[0, 3, 3, 3, 0] = 1.0
    y = conv.conv3d_fwd(x, w)
    # y[q0 - t + r] = w[t]
    for a in range(3):
        for bb in range(3):
            for c in range(3):
                assert np.allclose(y[0, 3 - a + 1, 3 - bb + 1, 3 - c + 1, :], w[:, a, bb, c, 0])
