"""Pins of the oracle's learned-guess march (the workload's learned initial
guess; Sec. 3, Phase 2 applied to the residual of a given guess).

* Mode 4 (a given guess, judged against the warm start, a kept guess
  projected in residual form) from a guess worse than the warm start is the
  warm start (mode 2) bit for bit, and from a guess better than it (the
  Richardson step) it projects the guess's own residual; mode 5 (the
  guess alone) from x_init = m^{n-1} is the warm start bit for bit.
* The residual-form projection meets its Galerkin condition with the seed's
  H_a:  V_a^T (r - A_seed (x0 - x_init)) = 0 for r = b - A_i x_init.
* ``network_inputs``: the residual planes are the step's residual at the
  image, b - A m^{n-1}, scaled to unit rms (checked against the oracle's
  operator), and a one-layer network passing them through turns the guess
  into the Richardson step m + dt (b - A m): the rms scale and the dt
  factor are pinned by it.
* A zero network is the warm start: the learned march without projection
  is the warm march, and with projection it reaches the plain trajectory.
"""
import numpy as np

from oracle import cnn_oracle as R
from paper_2511_17634_gb300 import synth


def _richardson_net():
    # channels (10, 1): the centre tap passes r_hat (its hi plane, and its lo
    # plane / 256), so net = r_hat and the guess is m + dt r, one Richardson
    # step from the warm start
    w = np.zeros((1, R.NIN, 3, 3))
    w[0, 8, 1, 1] = 1.0
    w[0, 9, 1, 1] = 1.0 / 256.0
    return R.flatten([(w, np.zeros(1))]), (R.NIN, 1)


def test_network_inputs_planes(orc):
    rng = np.random.default_rng(1)
    H, W, T, n, g2 = 4, 3, 1000, 250, 0.3
    mp, ms = rng.uniform(0, 1, size=(2, H * W)), rng.uniform(0, 1, size=(2, H * W))
    x, rho = R.network_inputs(mp, ms, n, T, g2, H, W)
    assert x.shape == (2, R.NIN, H * W)
    # hi planes are bfloat16 values, hi + lo/256 is the field to ~2^-17
    for k, m in ((0, mp), (2, ms)):
        assert np.array_equal(x[:, k], R.bf16(x[:, k]))
        assert np.abs(x[:, k] - m).max() <= 2.0 ** -8 * np.abs(m).max()
        assert np.abs(R.bf16(x[:, k]) + R.bf16(x[:, k + 1]) / 256 - m).max() <= 2.0 ** -16 * np.abs(m).max()
    # tau = 1/4: tau, 1 - tau, sin(pi/4), cos(pi/4)
    hq = np.sqrt(0.5)
    assert np.allclose(x[:, 4:8, 0], [[0.25, 0.75, hq, hq]] * 2, atol=1e-15)
    x0, _ = R.network_inputs(mp, ms, 1, T, g2, H, W)
    x1, _ = R.network_inputs(mp, ms, T, T, g2, H, W)
    assert np.all(np.abs(x0[0, [4, 5, 7], 0] - x1[0, [4, 5, 7], 0]) > 0.99)
    # the residual planes: the step's operator at timestep n, lagged on m,
    # applied to m itself, scaled to unit rms
    dt, h = 1.0 / T, 1.0 / H
    for k in range(2):
        C = orc.coeffs(H, W, g2, dt, h, mp[k])
        r = mp[k] / dt - orc.apply(H, W, C, mp[k])
        assert abs(rho[k] - np.linalg.norm(r) / np.sqrt(H * W)) <= 1e-12 * rho[k]
        rh = x[k, 8] + x[k, 9] / 256
        assert np.allclose(rh, r / rho[k], rtol=0, atol=1e-12)
        assert abs(np.mean(rh ** 2) - 1.0) <= 1e-12


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
    # the Richardson step m + dt r (residual well below the warm start's) is
    # kept and its own residual projected: the x0 residual equals that of
    # the projection computed here from the seed basis
    wl = synth.config(2, T=1000, ntargets=2)
    g = wl.groups[0]
    H, W = g.H, g.W
    n = 999
    dt, h, g2 = 1 / wl.T, 1 / H, float(wl.g2[n])
    ms0 = g.seeds.reshape(len(g.seeds), -1).copy()
    mt0 = g.targets.reshape(len(g.targets), -1).copy()
    p, ch = _richardson_net()
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




def test_richardson_network_gives_m_plus_dt_r(orc):
    wl = synth.config(2, T=1000, ntargets=3)
    g = wl.groups[0]
    H, W = g.H, g.W
    n = 1000
    dt, h, g2 = 1 / wl.T, 1 / H, float(wl.g2[n - 1])
    mp = g.targets.reshape(len(g.targets), -1)
    p, ch = _richardson_net()
    xg = R.learned_guess(p, ch, mp, mp, n, wl.T, g2, H, W)
    for k in range(len(mp)):
        C = orc.coeffs(H, W, g2, dt, h, mp[k])
        b = orc.rhs(H, W, dt, h, mp[k])
        r = b - orc.apply(H, W, C, mp[k])
        assert np.allclose(xg[k], mp[k] + dt * r, rtol=0, atol=1e-13)
        # the same with the network's BF16 operand rounding: hi + lo/256 of
        # r_hat keeps the step to a few 1e-5 of itself
        xb = R.learned_guess(p, ch, mp[k:k + 1], mp[k:k + 1], n, wl.T, g2, H, W, operand_round=R.bf16)[0]
        assert np.abs(xb - xg[k]).max() <= 1e-4 * np.abs(xg[k] - mp[k]).max()
        # dt A = I + dt K: the Richardson step leaves -dt K r, a fraction of r
        res = np.linalg.norm(b - orc.apply(H, W, C, xg[k])) / np.linalg.norm(r)
        assert res <= 0.35, (k, res)


def test_zero_network_learned_march_is_the_warm_march(orc):
    wl = synth.config(1, T=6)
    g = wl.groups[0]
    ch = (R.NIN, 4, 1)
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
