"""Pins of the FP64 CNN reference: finite differences, tap orientation, the
identity kernel, and Adam's first step."""
import numpy as np

from oracle import cnn_oracle as R


def test_identity_and_shift_kernels():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 1, 5, 4))
    w = np.zeros((1, 1, 3, 3))
    w[0, 0, 1, 1] = 1.0
    assert np.array_equal(R.conv(x, w, np.zeros(1)), x)
    w = np.zeros((1, 1, 3, 3))
    w[0, 0, 2, 1] = 1.0                          # di = +1: reads x[i+1, j]
    z = R.conv(x, w, np.zeros(1))
    assert np.array_equal(z[:, :, :-1, :], x[:, :, 1:, :]) and np.all(z[:, :, -1, :] == 0)
    w = np.zeros((1, 1, 3, 3))
    w[0, 0, 1, 0] = 1.0                          # dj = -1: reads x[i, j-1]
    z = R.conv(x, w, np.zeros(1))
    assert np.array_equal(z[:, :, :, 1:], x[:, :, :, :-1]) and np.all(z[:, :, :, 0] == 0)


def test_gradients_match_central_differences():
    rng = np.random.default_rng(2)
    ch = (3, 4, 2, 1)
    n = sum(co * ci * 9 + co for ci, co in zip(ch[:-1], ch[1:]))
    p = rng.normal(scale=0.4, size=n)
    x = rng.normal(size=(2, 3, 5, 6))
    t = rng.normal(size=(2, 1, 5, 6))
    loss, g = R.loss_and_grads(p, ch, x, t)
    h = 1e-6
    for k in rng.choice(n, 40, replace=False):
        e = np.zeros(n)
        e[k] = h
        fd = (R.loss_and_grads(p + e, ch, x, t)[0] - R.loss_and_grads(p - e, ch, x, t)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])


def test_adam_first_step_is_signed_lr():
    g = np.array([0.3, -2.0, 1e-3])
    p, m, v = R.adam(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    assert np.allclose(p, -0.01 * np.sign(g), rtol=1e-4)
