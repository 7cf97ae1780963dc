"""Pins of the FP64 CNN reference: finite differences, tap orientation, the
identity kernel, Adam over several steps (bias correction), and the BF16
operand rounding used to state the GPU kernels' error bound."""
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


def test_adam_bias_correction_over_three_steps():
    # Kingma & Ba 2015, Alg. 1 with lr = 0.1, beta1 = 0.9, beta2 = 0.999,
    # eps = 0, from p = m = v = 0 and the gradients g_1 = (1, -1/2, 2),
    # g_2 = (1/2, 1/2, -1), g_3 = (-1/4, 3/2, 1/2):
    #   m_t = b1 m_{t-1} + (1 - b1) g_t,  v_t = b2 v_{t-1} + (1 - b2) g_t^2,
    #   p_t = p_{t-1} - lr (m_t / (1 - b1^t)) / sqrt(v_t / (1 - b2^t)).
    # Worked out in exact rationals (square roots to 40 digits):
    #   t = 2: m = (7/50, 1/200, 2/25),  v = (1249, 1999/4, 4996) * 1e-6
    #   t = 3: m = (101/1000, 309/2000, 61/500),
    #          v = (1310251, 10997001/4, 5241004) * 1e-9
    expect = {
        1: [-0.1, 0.1, -0.1],
        2: [-1.932179638811409e-01, 9.473684210526316e-02, -1.266337039660403e-01],
        3: [-2.495841015354529e-01, 3.521237717292837e-02, -1.606766187869614e-01],
    }
    gs = [np.array([1.0, -0.5, 2.0]), np.array([0.5, 0.5, -1.0]), np.array([-0.25, 1.5, 0.5])]
    p, m, v = np.zeros(3), np.zeros(3), np.zeros(3)
    for t, g in enumerate(gs, 1):
        p, m, v = R.adam(p, g, m, v, t, lr=0.1, b1=0.9, b2=0.999, eps=0.0)
        assert np.allclose(p, expect[t], rtol=1e-13, atol=0), (t, p)
    assert np.allclose(m, [0.101, 0.1545, 0.122], rtol=1e-14)
    assert np.allclose(v, [1.310251e-3, 2.74925025e-3, 5.241004e-3], rtol=1e-14)


def test_bf16_rounding_is_nearest_even_on_8_bits():
    # bfloat16 keeps 8 significant bits: spacing 2^-7 on [1, 2)
    u = 2.0 ** -7
    vals = np.array([1.0, 1 + u / 2, 1 + 3 * u / 2, 1 + u / 2 + 2 ** -20, -(1 + 3 * u / 2), 3.0e-39,
                     65504.0, 0.0])
    want = np.array([1.0, 1.0, 1 + 2 * u, 1 + u, -(1 + 2 * u), R.bf16(3.0e-39), 65536.0, 0.0])
    got = R.bf16(vals)
    assert np.array_equal(got[:5], want[:5])          # ties to even, sign symmetric
    assert got[6] == 65536.0 and got[7] == 0.0          # 65504 = 2^16 - 32 rounds up
    # every value is a bfloat16: its float32 bits have a zero low half
    bits = got.astype(np.float32).view(np.uint32)
    assert np.all(bits & 0xFFFF == 0)
    x = np.random.default_rng(3).normal(size=1000)
    # unit roundoff of 8 significant bits: half an ulp, 2^-8 relative
    assert np.all(np.abs(R.bf16(x) - x) <= 2.0 ** -8 * np.abs(x))


def test_operand_rounding_hook_is_exact_when_identity():
    rng = np.random.default_rng(4)
    ch = (2, 3, 1)
    n = sum(co * ci * 9 + co for ci, co in zip(ch[:-1], ch[1:]))
    p = rng.normal(size=n)
    x = rng.normal(size=(2, 2, 4, 5))
    t = rng.normal(size=(2, 1, 4, 5))
    l0, g0 = R.loss_and_grads(p, ch, x, t)
    l1, g1 = R.loss_and_grads(p, ch, x, t, operand_round=lambda a: a)
    assert l0 == l1 and np.array_equal(g0, g1)
    # rounding changes the result by about the BF16 unit (2^-8) times the
    # condition of the sums, not more
    l2, g2 = R.loss_and_grads(p, ch, x, t, operand_round=R.bf16)
    assert 0 < np.linalg.norm(g2 - g0) <= 5e-2 * np.linalg.norm(g0)
