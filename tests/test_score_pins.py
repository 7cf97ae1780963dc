"""Pins of the oracle's score extraction and probability-flow embedding (end
of Sec. 2.3, Sec. 4.1) against closed forms."""
import numpy as np
import pytest


def _grid(H, W):
    i, j = np.meshgrid(np.arange(W), np.arange(H), indexing="ij")   # p = i*H + j
    return i.astype(float), j.astype(float)


def test_central_difference_is_exact_on_quadratics(orc):
    # interior points: (m(x+h) - m(x-h)) / 2h is the exact derivative of a
    # quadratic in x = i h, y = j h; a dropped 1/h, a factor 2 or a swapped
    # axis fails here
    H, W = 7, 9
    h = 1.0 / H
    i, j = _grid(H, W)
    x, y = i * h, j * h
    m = 0.7 * x * x - 1.3 * y * y + 0.4 * x * y + 2.0 * x - 0.5 * y + 0.1
    sx, sy = orc.score(H, W, h, m.ravel())
    sx, sy = sx.reshape(W, H), sy.reshape(W, H)
    gx = 1.4 * x + 0.4 * y + 2.0
    gy = -2.6 * y + 0.4 * x - 0.5
    inner = (slice(1, W - 1), slice(1, H - 1))
    assert np.allclose(sx[inner], gx[inner], rtol=0, atol=1e-12)
    assert np.allclose(sy[inner], gy[inner], rtol=0, atol=1e-12)


def test_zero_padding_at_the_border(orc):
    H, W = 5, 4
    h = 0.25
    m = np.arange(H * W, dtype=float) + 1.0
    sx, sy = orc.score(H, W, h, m)
    M = m.reshape(W, H)
    # west column: the missing neighbour is zero; north row likewise
    assert np.allclose(sx.reshape(W, H)[0], M[1] / (2 * h))
    assert np.allclose(sx.reshape(W, H)[W - 1], -M[W - 2] / (2 * h))
    assert np.allclose(sy.reshape(W, H)[:, 0], M[:, 1] / (2 * h))
    assert np.allclose(sy.reshape(W, H)[:, H - 1], -M[:, H - 2] / (2 * h))


def test_orientation_x_is_the_column_index(orc):
    # a field varying only with the column index i (x, east-west) has no y score
    H, W = 6, 8
    h = 1.0 / H
    i, _ = _grid(H, W)
    sx, sy = orc.score(H, W, h, (3.0 * i * h).ravel())
    inner = (slice(1, W - 1), slice(1, H - 1))
    assert np.allclose(sx.reshape(W, H)[inner], 3.0)
    assert np.allclose(sy.reshape(W, H)[inner], 0.0)


def test_embedding_accumulates_forward_euler_steps(orc):
    # constant scores: x^n = -dt/2 * sum_k g2_k * s exactly
    N = 11
    rng = np.random.default_rng(0)
    sx, sy = rng.normal(size=N), rng.normal(size=N)
    ex, ey = np.zeros(N), np.zeros(N)
    g2 = [0.1, 0.2, 0.35]
    dt = 0.01
    for g in g2:
        orc.embed_step(dt, g, sx, sy, ex, ey)
    assert np.allclose(ex, -0.5 * dt * sum(g2) * sx, rtol=1e-14, atol=0)
    assert np.allclose(ey, -0.5 * dt * sum(g2) * sy, rtol=1e-14, atol=0)


def test_march_scores_are_the_scores_of_the_march(orc):
    # march_scores returns the march's own states and their scores, and the
    # embedding uses grad m^{n-1} with (g^{n-1})^2
    from paper_2511_17634_gb300 import synth
    wl = synth.config(1, T=6)
    g = wl.groups[0]
    ms, mt, S, E = orc.march_scores(g.H, g.W, wl.T, wl.g2, g.seeds, g.targets, g.target_seed,
                                    steps=3, tol_ref=1e-12)
    _, mt2, _ = orc.march(g.H, g.W, wl.T, wl.g2, g.seeds, g.targets, g.target_seed, steps=3,
                          tol_ref=1e-12)
    assert np.array_equal(mt, mt2)
    h = 1.0 / g.H
    for k in range(len(mt)):
        assert np.array_equal(S[-1, k, 0], orc.score(g.H, g.W, h, mt[k])[0])
    # step 1 used the images' scores with (g^1)^2, steps 2-3 the scores of m^1, m^2
    dt = 1.0 / wl.T
    m0 = g.targets.reshape(len(g.targets), -1)
    ref = -0.5 * dt * wl.g2[0] * orc.score(g.H, g.W, h, m0[0])[0]
    ref = ref - 0.5 * dt * wl.g2[0] * S[0, 0, 0] - 0.5 * dt * wl.g2[1] * S[1, 0, 0]
    assert np.allclose(E[0, 0], ref, rtol=1e-13, atol=1e-15)
