"""Pins of the oracle's learned-guess march (the workload's learned initial
guess; Sec. 3, Phase 2 applied to the residual of a given guess).

* Mode 4 (a given guess, judged against the warm start, a kept guess
  projected in residual form) from a guess worse than the warm start is the
  warm start (mode 2) bit for bit, and from a guess better than it (the
  explicit Euler step) it projects the guess's own residual; mode 5 (the
  guess alone) from x_init = m^{n-1} is the warm start bit for bit.
* The residual-form projection meets its Galerkin condition with the seed's
  H_a:  V_a^T (r - A_seed (x0 - x_init)) = 0 for r = b - A_i x_init.
* ``learned_guess``: a one-layer network holding half the five-point pixel
  Laplacian on the m^{n-1} plane turns the guess into the explicit Euler
  step m + (s_n / 2) L m of the linear part (s_n = dt g^2 / h^2), computed
  here with numpy, which leaves about a quarter of the warm start's
  residual -- half or twice the scale leave about half or more.
* A zero network is the warm start: the learned march without projection
  is the warm march, and with projection it reaches the plain trajectory.
"""
import numpy as np

from oracle import cnn_oracle as R
from paper_2511_17634_gb300 import synth


def _laplace_net():
    # channels (8, 1): tap [di+1][dj+1] multiplies m[i+di, j+dj]; half the
    # pixel Laplacian on the hi plane and on the lo plane / 256 acts on m
    L = 0.5 * np.array([[0, 1, 0], [1, -4, 1], [0, 1, 0]], dtype=float)
    w = np.zeros((1, 8, 3, 3))
    w[0, 0] = L
    w[0, 1] = L / 256.0
    return R.flatten([(w, np.zeros(1))]), (8, 1)


def test_network_inputs_plane_order_and_time_planes():
    rng = np.random.default_rng(1)
    mp, ms = rng.uniform(0, 1, size=(2, 12)), rng.uniform(0, 1, size=(2, 12))
    x = R.network_inputs(mp, ms, 250, 1000)
    assert x.shape == (2, 8, 12)
    # hi planes are bfloat16 values, hi + lo/256 is the field to ~2^-17
    for k, m in ((0, mp), (2, ms)):
        assert np.array_equal(x[:, k], R.bf16(x[:, k]))
        assert np.abs(x[:, k] - m).max() <= 2.0 ** -8 * np.abs(m).max()
        assert np.abs(R.bf16(x[:, k]) + R.bf16(x[:, k + 1]) / 256 - m).max() <= 2.0 ** -16 * np.abs(m).max()
    # tau = 1/4: tau, 1 - tau, sin(pi/4), cos(pi/4)
    h = np.sqrt(0.5)
    assert np.allclose(x[:, 4:, 0], [[0.25, 0.75, h, h]] * 2, atol=1e-15)
    # the first and the last timestep are told apart on every time plane
    # but the sine
    x0, x1 = R.network_inputs(mp, ms, 1, 1000), R.network_inputs(mp, ms, 1000, 1000)
    assert np.all(np.abs(x0[0, [4, 5, 7], 0] - x1[0, [4, 5, 7], 0]) > 0.99)
    assert R.guess_scale(1000, 0.02, 32) == 0.02 * 1024 / 1000


def test_guess_modes_reduce_to_projection_and_warm_start(orc):
    wl = synth.config(2, T=1000, ntargets=5)
    g = wl.groups[0]
    H, W = g.H, g.W
    n = 600
    ms0 = g.seeds.reshape(len(g.seeds), -1).copy()
    mt0 = g.targets.reshape(len(g.targets), -1).copy()
    out = {}
    for name, mode, xi in (("zero_guess", orc.MODE_GUESS_PROJECTED, np.zeros_like(mt0)),
                           ("warm_guess", orc.MODE_GUESS_PROJECTED, mt0.copy()),
                           ("warm", orc.MODE_WARM, None),
                           ("guess_warm", orc.MODE_GUESS, mt0.copy())):
        ms, mt = ms0.copy(), mt0.copy()
        st = orc.march_step(H, W, 1 / wl.T, 1 / H, float(wl.g2[n]), ms, mt, g.target_seed, mode=mode,
                            xinit=xi, tol_ref=1e-10)
        out[name] = (mt, st)
    # x_init = 0 leaves the residual b, far above the warm start's: the judge
    # falls back to the warm start, which is then mode 2 exactly
    for name in ("zero_guess", "guess_warm"):
        assert np.array_equal(out["warm"][0], out[name][0])
        assert np.array_equal(out["warm"][1].tgt_iters, out[name][1].tgt_iters)
        assert np.array_equal(out["warm"][1].tgt_x0res, out[name][1].tgt_x0res)
    # a guess equal to the warm start is kept (the judge wants strictly less)
    # and projected: less residual than the warm start alone
    assert (out["warm_guess"][1].tgt_x0res < out["warm"][1].tgt_x0res).all()


def test_judge_keeps_a_guess_better_than_the_warm_start(orc):
    # the explicit Euler step (residual ~1/4 of the warm start's) is kept and
    # its own residual projected: the x0 residual equals that of the
    # projection computed here from the seed basis
    wl = synth.config(2, T=1000, ntargets=2)
    g = wl.groups[0]
    H, W = g.H, g.W
    n = 999
    dt, h, g2 = 1 / wl.T, 1 / H, float(wl.g2[n])
    ms0 = g.seeds.reshape(len(g.seeds), -1).copy()
    mt0 = g.targets.reshape(len(g.targets), -1).copy()
    p, ch = _laplace_net()
    xi = R.learned_guess(p, ch, mt0, mt0, n + 1, wl.T, g2, H, W)
    ms, mt = ms0.copy(), mt0.copy()
    st = orc.march_step(H, W, dt, h, g2, ms, mt, g.target_seed, mode=orc.MODE_GUESS_PROJECTED, xinit=xi,
                        a=12, fixed_a=True, tol_ref=1e-10)
    for k in range(len(mt0)):
        s = int(g.target_seed[k])
        Cs = orc.coeffs(H, W, g2, dt, h, ms0[s])
        r0 = orc.gmres(H, W, Cs, orc.rhs(H, W, dt, h, ms0[s]), tol=1e-10, m=40, maxit=1000, capture=12,
                       fixed=True)
        Ci = orc.coeffs(H, W, g2, dt, h, mt0[k])
        b = orc.rhs(H, W, dt, h, mt0[k])
        r = b - orc.apply(H, W, Ci, xi[k])
        assert np.linalg.norm(r) < np.linalg.norm(b - orc.apply(H, W, Ci, mt0[k]))
        x0, _ = orc.project(r0.V, r0.Hbar, r0.a, r0.has_next, r, xinit=xi[k])
        res0 = np.linalg.norm(b - orc.apply(H, W, Ci, x0)) / np.linalg.norm(b)
        assert abs(st.tgt_x0res[k] - res0) <= 1e-12 * res0


def test_residual_form_projection_galerkin_condition(orc):
    wl = synth.config(2, T=1000, ntargets=3)
    g = wl.groups[0]
    H, W = g.H, g.W
    dt, h, g2 = 1 / wl.T, 1 / H, float(wl.g2[800])
    s0 = g.seeds[int(g.target_seed[0])].reshape(-1)
    Cs = orc.coeffs(H, W, g2, dt, h, s0)
    r0 = orc.gmres(H, W, Cs, orc.rhs(H, W, dt, h, s0), tol=1e-10, m=40, maxit=400, capture=12,
                   fixed=True)
    mt = g.targets[0].reshape(-1)
    Ci = orc.coeffs(H, W, g2, dt, h, mt)
    b = orc.rhs(H, W, dt, h, mt)
    xi = mt + 0.01 * np.random.default_rng(2).normal(size=H * W)
    r = b - orc.apply(H, W, Ci, xi)
    x0, lsq = orc.project(r0.V, r0.Hbar, r0.a, r0.has_next, r, xinit=xi)
    assert not lsq
    gal = r0.V[:r0.a] @ (r - orc.apply(H, W, Cs, x0 - xi))
    assert np.abs(gal).max() <= 1e-11 * np.linalg.norm(r)


def test_laplacian_network_gives_the_explicit_euler_guess(orc):
    wl = synth.config(2, T=1000, ntargets=3)
    g = wl.groups[0]
    H, W, N = g.H, g.W, g.N
    n = 1000
    dt, h, g2 = 1 / wl.T, 1 / H, float(wl.g2[n - 1])
    mp = g.targets.reshape(len(g.targets), -1)
    p, ch = _laplace_net()
    xg = R.learned_guess(p, ch, mp, mp, n, wl.T, g2, H, W)
    s = dt * g2 / (h * h)
    for k in range(len(mp)):
        m = mp[k].reshape(W, H)
        mpad = np.pad(m, 1)
        lap = mpad[2:, 1:-1] + mpad[:-2, 1:-1] + mpad[1:-1, 2:] + mpad[1:-1, :-2] - 4 * m
        assert np.allclose(xg[k], (m + 0.5 * s * lap).reshape(-1), rtol=0, atol=1e-13)
        # the same with the network's BF16 operand rounding: hi + lo/256
        # keeps the Laplacian to a few 1e-5 of itself (one plane would not)
        xb = R.learned_guess(p, ch, mp[k:k + 1], mp[k:k + 1], n, wl.T, g2, H, W, operand_round=R.bf16)[0]
        assert np.abs(xb - xg[k]).max() <= 1e-4 * np.abs(xg[k] - mp[k]).max()
        C = orc.coeffs(H, W, g2, dt, h, mp[k])
        b = orc.rhs(H, W, dt, h, mp[k])
        res_guess = np.linalg.norm(b - orc.apply(H, W, C, xg[k]))
        res_warm = np.linalg.norm(b - orc.apply(H, W, C, mp[k]))
        # ~0.25 at the right scale (the nonlinear term is left); half or
        # twice the scale leaves ~0.47 and ~1.2 of the warm residual
        assert res_guess <= 0.35 * res_warm, (k, res_guess / res_warm)


def test_zero_network_learned_march_is_the_warm_march(orc):
    wl = synth.config(1, T=6)
    g = wl.groups[0]
    ch = (8, 4, 1)
    p = np.zeros(sum(co * ci * 9 + co for ci, co in zip(ch[:-1], ch[1:])))
    kw = dict(m_seed=30, a=30, m_ref=30, tol_ref=1e-12)
    _, warm, _ = orc.march(g.H, g.W, wl.T, wl.g2, g.seeds, g.targets, g.target_seed,
                           mode=orc.MODE_WARM, **kw)
    _, plain, _ = orc.march(g.H, g.W, wl.T, wl.g2, g.seeds, g.targets, g.target_seed,
                            mode=orc.MODE_PLAIN, **kw)
    _, lw, _ = orc.march_learned(g.H, g.W, wl.T, wl.g2, g.seeds, g.targets, g.target_seed, p, ch,
                                 project=False, **kw)
    assert np.array_equal(lw, warm)
    _, lp, st = orc.march_learned(g.H, g.W, wl.T, wl.g2, g.seeds, g.targets, g.target_seed, p, ch,
                                  project=True, **kw)
    assert all((s.tgt_status == 0).all() for s in st)
    assert np.abs(lp - plain).max() <= 1e-9 * np.abs(plain).max()
