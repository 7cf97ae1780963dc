"""Pins of the FP64 CPU oracle against facts fixed by the paper and by
mathematics, not against itself.

* The five-point system (Sec. 2.3, Eq. 11 and its coefficient listing) must
  reproduce the linearised log-density Fokker-Planck operator (Eq. 5 with the
  semi-explicit <grad m~, grad m> term) exactly on quadratic fields, where
  central differences and the five-point Laplacian have no truncation error.
* Zero padding (Sec. 2.3) must equal embedding the grid in a larger grid with
  a ring of zeros.
* The CSR matrix assembled from the block form (Eq. 12-15) must equal the
  stencil, and have that block structure.
* GMRES must match a dense LU solve and the discrete-sine closed form of the
  shifted Dirichlet Laplacian, and satisfy the Arnoldi identities and the FOM
  residual formula (Saad 2003, Prop. 6.7) that the Galerkin projection of
  Sec. 3 relies on.
"""
import numpy as np
import pytest

from paper_2511_17634_gb300 import synth


def _grid(W, H, h):
    x = (np.arange(W) * h)[:, None] * np.ones((1, H))
    y = np.ones((W, 1)) * (np.arange(H) * h)[None, :]
    return x, y


def _quad(coef, x, y):
    a0, a1, a2, a3, a4, a5 = coef
    f = a0 + a1 * x + a2 * y + a3 * x * x + a4 * x * y + a5 * y * y
    fx = a1 + 2 * a3 * x + a4 * y
    fy = a2 + a4 * x + 2 * a5 * y
    lap = 2 * a3 + 2 * a5
    return f, fx, fy, lap


@pytest.mark.parametrize("W,H", [(7, 5), (6, 9)])
def test_stencil_reproduces_linearised_pde_on_quadratics(orc, W, H):
    rng = np.random.default_rng(11)
    h, dt, g2 = 0.1, 0.5, 0.3
    x, y = _grid(W, H, h)
    u, ux, uy, ulap = _quad(rng.normal(size=6), x, y)
    mt, mtx, mty, _ = _quad(rng.normal(size=6), x, y)
    fxc, fyc = rng.normal(size=6), rng.normal(size=6)
    fx, fxx, _, _ = _quad(fxc, x, y)
    fy, _, fyy, _ = _quad(fyc, x, y)
    C = orc.coeffs(H, W, g2, dt, h, mt, fx, fy)
    Au = orc.apply(H, W, C, u).reshape(W, H)
    # Eq. (5) linearised, moved to the left: m/dt + f.grad m - g^2/2 lap m - g^2/2 grad m~ . grad m
    expect = (u / dt + fx * ux + fy * uy - 0.5 * g2 * ulap
              - 0.5 * g2 * (mtx * ux + mty * uy))
    inner = (slice(1, W - 1), slice(1, H - 1))
    scale = np.abs(u / dt).max() + np.abs(expect).max()
    assert np.abs(Au[inner] - expect[inner]).max() <= 1e-12 * scale
    # right-hand side: b = m^{n-1}/dt - Div f
    b = orc.rhs(H, W, dt, h, u, fx, fy).reshape(W, H)
    expect_b = u / dt - (fxx + fyy)
    assert np.abs(b[inner] - expect_b[inner]).max() <= 1e-12 * scale


def test_constant_field_rows_sum_to_inverse_dt(orc):
    # f = 0: the Laplacian and gradient of a constant vanish, so every interior
    # row of A sums to 1/dt whatever m~ is.
    rng = np.random.default_rng(2)
    H, W, dt, h, g2 = 6, 8, 0.01, 1 / 6, 0.02
    C = orc.coeffs(H, W, g2, dt, h, rng.uniform(0, 1, H * W))
    Au = orc.apply(H, W, C, np.ones(H * W)).reshape(W, H)
    assert np.allclose(Au[1:-1, 1:-1], 1 / dt, rtol=1e-14, atol=0)
    assert np.all(Au[0, :] > 1 / dt) and np.all(Au[:, -1] > 1 / dt)


def test_zero_padding_equals_zero_ring_embedding(orc):
    rng = np.random.default_rng(3)
    H, W, dt, h, g2 = 5, 4, 0.02, 0.2, 0.7
    u, mt, fx, fy = (rng.normal(size=(W, H)) for _ in range(4))

    def pad(a):
        out = np.zeros((W + 2, H + 2))
        out[1:-1, 1:-1] = a
        return out

    C = orc.coeffs(H, W, g2, dt, h, mt, fx, fy)
    small = orc.apply(H, W, C, u).reshape(W, H)
    Cb = orc.coeffs(H + 2, W + 2, g2, dt, h, pad(mt), pad(fx), pad(fy))
    big = orc.apply(H + 2, W + 2, Cb, pad(u)).reshape(W + 2, H + 2)[1:-1, 1:-1]
    assert np.allclose(small, big, rtol=1e-14, atol=1e-12)
    bs = orc.rhs(H, W, dt, h, u, fx, fy).reshape(W, H)
    bb = orc.rhs(H + 2, W + 2, dt, h, pad(u), pad(fx), pad(fy)).reshape(W + 2, H + 2)[1:-1, 1:-1]
    assert np.allclose(bs, bb, rtol=1e-14, atol=1e-12)


def test_csr_block_form_matches_stencil(orc):
    rng = np.random.default_rng(4)
    H, W = 5, 7
    C = orc.coeffs(H, W, 0.4, 0.1, 0.25, rng.normal(size=H * W), rng.normal(size=H * W),
                   rng.normal(size=H * W))
    A = orc.csr_dense(H, W, C)
    x = rng.normal(size=H * W)
    assert np.allclose(A @ x, orc.apply(H, W, C, x), rtol=1e-14, atol=1e-12)
    rp, col, val = orc.csr(H, W, C)
    assert np.allclose(orc.csr_matvec(rp, col, val, x), A @ x, rtol=1e-14, atol=1e-12)
    # block structure: W x W blocks of H x H; M tridiagonal, L/U diagonal, rest 0
    for bi in range(W):
        for bj in range(W):
            blk = A[bi * H:(bi + 1) * H, bj * H:(bj + 1) * H]
            if bi == bj:
                assert np.all(np.triu(blk, 2) == 0) and np.all(np.tril(blk, -2) == 0)
                assert np.all(np.diag(blk) == C[bi * H:(bi + 1) * H, 0])
                assert np.all(np.diag(blk, 1) == C[bi * H:(bi + 1) * H - 1, 3])   # north
                assert np.all(np.diag(blk, -1) == C[bi * H + 1:(bi + 1) * H, 4])  # south
            elif bj == bi + 1:
                assert np.all(blk == np.diag(C[bi * H:(bi + 1) * H, 1]))          # east (U)
            elif bj == bi - 1:
                assert np.all(blk == np.diag(C[bi * H:(bi + 1) * H, 2]))          # west (L)
            else:
                assert np.all(blk == 0)


def test_m_matrix_bound(orc):
    # f = 0 and |m~_{+} - m~_{-}| <= 4: off-diagonals <= 0, A 1 >= 1/dt, hence
    # ||A^{-1}||_inf <= dt.
    rng = np.random.default_rng(5)
    H, W, dt, h, g2 = 7, 6, 0.01, 1 / 7, 0.5
    mt = rng.uniform(0, 1.9, H * W)
    C = orc.coeffs(H, W, g2, dt, h, mt)
    A = orc.csr_dense(H, W, C)
    off = A - np.diag(np.diag(A))
    assert off.max() <= 0
    inv = np.linalg.inv(A)
    assert inv.min() >= -1e-15
    assert np.abs(inv).sum(axis=1).max() <= dt * (1 + 1e-12)


@pytest.mark.parametrize("H,W", [(3, 3), (4, 4), (3, 5), (8, 8)])
def test_gmres_matches_dense_lu(orc, H, W):
    rng = np.random.default_rng(6 + H * W)
    dt, h, g2 = 0.01, 1 / H, 0.25
    mt = rng.uniform(0, 1, H * W)
    C = orc.coeffs(H, W, g2, dt, h, mt, rng.normal(size=H * W), rng.normal(size=H * W))
    A = np.stack([orc.apply(H, W, C, e) for e in np.eye(H * W)], axis=1)
    b = rng.normal(size=H * W)
    x_np = np.linalg.solve(A, b)
    x_lu = orc.dense_lu_solve(A, b)
    assert np.linalg.norm(x_lu - x_np) <= 1e-13 * np.linalg.norm(x_np)
    r = orc.gmres(H, W, C, b, tol=1e-14, m=5, maxit=500)
    assert r.status == 0
    assert np.linalg.norm(r.x - x_np) <= 1e-12 * np.linalg.norm(x_np)


def test_gmres_matches_discrete_sine_closed_form(orc):
    # m~ = 0, f = 0: A = (1/dt) I + c (5-point Dirichlet negative Laplacian)
    # with eigenvectors sin(p pi (i+1)/(W+1)) sin(q pi (j+1)/(H+1)).
    H, W, T = 6, 9, 100
    dt, h, g2 = 1 / T, 1 / H, 0.25
    c = g2 / (2 * h * h)
    rng = np.random.default_rng(7)
    B = rng.normal(size=(W, H))
    SW = np.sqrt(2 / (W + 1)) * np.sin(np.pi * np.outer(np.arange(1, W + 1), np.arange(1, W + 1)) / (W + 1))
    SH = np.sqrt(2 / (H + 1)) * np.sin(np.pi * np.outer(np.arange(1, H + 1), np.arange(1, H + 1)) / (H + 1))
    lw = 2 * c * (1 - np.cos(np.pi * np.arange(1, W + 1) / (W + 1)))
    lh = 2 * c * (1 - np.cos(np.pi * np.arange(1, H + 1) / (H + 1)))
    lam = 1 / dt + lw[:, None] + lh[None, :]
    X = SW @ ((SW @ B @ SH) / lam) @ SH
    C = orc.coeffs(H, W, g2, dt, h, np.zeros(H * W))
    r = orc.gmres(H, W, C, B.reshape(-1), tol=1e-14, m=20, maxit=500)
    assert r.status == 0
    assert np.linalg.norm(r.x - X.reshape(-1)) <= 1e-12 * np.linalg.norm(X)


def test_g_zero_gives_identity_step(orc):
    H, W, dt = 5, 6, 0.02
    rng = np.random.default_rng(8)
    mprev = rng.uniform(0, 1, H * W)
    C = orc.coeffs(H, W, 0.0, dt, 1 / H, mprev)
    b = orc.rhs(H, W, dt, 1 / H, mprev)
    r = orc.gmres(H, W, C, b, tol=1e-12, m=10, maxit=50)
    assert r.iters == 1 and r.status == 0
    assert np.allclose(r.x, mprev, rtol=1e-15, atol=1e-15)


def _hard_system(orc, H=16, W=16, seed=9):
    # the paper's own setting (g = 0.5, T = 100) conditions the system worse
    # than the linear-beta schedule, so GMRES needs more than a handful of steps
    img = synth.config(1).groups[0].seeds[0][:W, :H]
    dt, h, g2 = 1 / 100, 1 / H, 0.25
    mt = np.ascontiguousarray(img).reshape(-1)
    C = orc.coeffs(H, W, g2, dt, h, mt)
    b = orc.rhs(H, W, dt, h, mt)
    A = np.stack([orc.apply(H, W, C, e) for e in np.eye(H * W)], axis=1)
    return C, b, A


def test_arnoldi_identities(orc):
    H = W = 16
    C, b, A = _hard_system(orc)
    a = 8
    r = orc.gmres(H, W, C, b, tol=1e-13, m=40, maxit=400, capture=a)
    assert r.status == 0 and r.iters > a
    assert r.a == a and r.has_next == 1
    V = r.V.T                      # N x (a+1)
    assert np.abs(V.T @ V - np.eye(a + 1)).max() <= 1e-13
    normA = np.linalg.norm(A, 2)
    assert np.linalg.norm(A @ V[:, :a] - V @ r.Hbar) <= 1e-13 * normA
    # V_a^T A V_a = H_a (the projected seed matrix of Sec. 3, Phase 2)
    assert np.abs(V[:, :a].T @ A @ V[:, :a] - r.Hbar[:a]).max() <= 1e-12 * normA
    # v_1 = b / ||b||
    assert np.allclose(V[:, 0], b / np.linalg.norm(b), rtol=0, atol=1e-15)


def test_gmres_residuals_monotone(orc):
    H = W = 16
    C, b, A = _hard_system(orc)
    r = orc.gmres(H, W, C, b, tol=1e-12, m=5, maxit=400)
    assert r.status == 0
    hst = r.hist
    assert np.all(np.diff(hst) <= 1e-12 * hst[:-1])
    true = np.linalg.norm(b - A @ r.x) / np.linalg.norm(b)
    assert abs(true - r.rel_res) <= 1e-12
    assert r.rel_res <= 1e-12


def test_projection_of_seed_is_fom_iterate(orc):
    # target == seed: x0 = V_a H_a^{-1} V_a^T b is the FOM iterate, whose
    # residual is -h_{a+1,a} (e_a^T alpha) v_{a+1} (Saad 2003, Prop. 6.7).
    H = W = 16
    C, b, A = _hard_system(orc)
    a = 5
    r = orc.gmres(H, W, C, b, tol=1e-13, m=40, maxit=400, capture=a)
    x0, lsq = orc.project(r.V, r.Hbar, r.a, r.has_next, b)
    assert not lsq
    alpha = np.linalg.solve(r.Hbar[:a], r.V[:a] @ b)
    res = b - A @ x0
    expect = r.Hbar[a, a - 1] * abs(alpha[-1])
    assert abs(np.linalg.norm(res) - expect) <= 1e-10 * expect
    cosang = abs(res @ r.V[a]) / np.linalg.norm(res)
    assert cosang >= 1 - 1e-10
    # Galerkin condition: V_a^T (b - A x0) = 0
    assert np.abs(r.V[:a] @ res).max() <= 1e-12 * np.linalg.norm(b)


def test_exact_recovery_when_seed_converges_in_first_cycle(orc):
    wl = synth.config(1)
    g = wl.groups[0]
    H, W, T = g.H, g.W, wl.T
    mt = np.ascontiguousarray(g.seeds[0]).reshape(-1)
    C = orc.coeffs(H, W, wl.g2[T - 1], 1 / T, 1 / H, mt)
    b = orc.rhs(H, W, 1 / T, 1 / H, mt)
    r = orc.gmres(H, W, C, b, tol=1e-10, m=30, maxit=300, capture=30)
    assert r.status == 0 and r.a == r.iters < 30
    V = r.V.T
    assert np.abs(V.T @ V - np.eye(V.shape[1])).max() <= 1e-13
    x0, _ = orc.project(r.V, r.Hbar, r.a, r.has_next, b)
    ref = orc.gmres(H, W, C, b, x0=x0, tol=1e-8, m=30, maxit=300)
    assert ref.iters == 0 and ref.rel_res <= 1e-8
    assert np.linalg.norm(x0 - r.x) <= 1e-9 * np.linalg.norm(r.x)


def test_projection_least_squares_fallback(orc):
    # A numerically singular H_a switches the projection to
    # min || Hbar alpha - V_{a+1}^T r || (reading of Sec. 3 for that case).
    rng = np.random.default_rng(12)
    N, a = 40, 4
    Q, _ = np.linalg.qr(rng.normal(size=(N, a + 1)))
    Hb = np.triu(rng.normal(size=(a + 1, a)), -1)
    Hb[:a, a - 1] = Hb[:a, : a - 1] @ rng.normal(size=a - 1)   # H_a singular ...
    Hb[a, a - 1] = 1.0                                          # ... Hbar full rank
    r = rng.normal(size=N)
    x0, lsq = orc.project(Q.T.copy(), Hb, a, 1, r)
    assert lsq
    alpha, *_ = np.linalg.lstsq(Hb, Q.T @ r, rcond=None)
    assert np.allclose(x0, Q[:, :a] @ alpha, rtol=1e-10, atol=1e-12)
    # non-singular case: Givens QR solve equals a dense solve of H_a
    Hb2 = np.triu(rng.normal(size=(a + 1, a)), -1) + 3 * np.eye(a + 1, a)
    x1, lsq1 = orc.project(Q.T.copy(), Hb2, a, 1, r, xinit=np.ones(N))
    assert not lsq1
    al2 = np.linalg.solve(Hb2[:a], Q[:, :a].T @ r)
    assert np.allclose(x1, 1 + Q[:, :a] @ al2, rtol=1e-12, atol=1e-12)


def test_solve_is_linear_and_transpose_symmetric(orc):
    rng = np.random.default_rng(13)
    H, W, dt, g2 = 12, 9, 0.01, 0.25
    h = 1 / H
    mt = rng.uniform(0, 1, (W, H))
    C = orc.coeffs(H, W, g2, dt, h, mt)
    b1, b2 = rng.normal(size=H * W), rng.normal(size=H * W)
    s = lambda bb: orc.gmres(H, W, C, bb, tol=1e-14, m=30, maxit=600).x
    x12 = s(b1 + b2)
    assert np.linalg.norm(x12 - s(b1) - s(b2)) <= 1e-12 * np.linalg.norm(x12)
    # f = 0: exchanging x and y maps the operator onto itself, so the
    # transposed image's solution is the transposed solution.
    Ct = orc.coeffs(W, H, g2, dt, h, mt.T.copy())
    xt = orc.gmres(W, H, Ct, b1.reshape(W, H).T.copy(), tol=1e-14, m=30, maxit=600).x
    assert np.allclose(xt.reshape(H, W).T, s(b1).reshape(W, H), rtol=0,
                       atol=1e-12 * np.abs(s(b1)).max())


def test_march_modes_reach_same_trajectory(orc):
    wl = synth.config(1, T=8)
    g = wl.groups[0]
    out = {}
    for mode in (orc.MODE_PROJECTED, orc.MODE_PLAIN, orc.MODE_WARM):
        ms, mt, st = orc.march(g.H, g.W, wl.T, wl.g2, g.seeds, g.targets, g.target_seed,
                               mode=mode, m_seed=30, a=30, m_ref=30, tol_ref=1e-12)
        assert all((s.tgt_status == 0).all() and (s.tgt_res <= 1e-12).all() for s in st)
        out[mode] = mt
    ref = out[orc.MODE_PLAIN]
    for mode in (orc.MODE_PROJECTED, orc.MODE_WARM):
        assert np.abs(out[mode] - ref).max() <= 1e-9 * np.abs(ref).max()


def test_march_step_equals_seed_gmres(orc):
    # the seed update inside one march step is a plain GMRES solve from 0
    wl = synth.config(1, T=4)
    g = wl.groups[0]
    H, W = g.H, g.W
    ms = g.seeds.reshape(1, -1).copy()
    mt = g.targets.reshape(len(g.targets), -1).copy()
    m0 = ms[0].copy()
    orc.march_step(H, W, 1 / wl.T, 1 / H, wl.g2[0], ms, mt, g.target_seed)
    C = orc.coeffs(H, W, wl.g2[0], 1 / wl.T, 1 / H, m0)
    r = orc.gmres(H, W, C, orc.rhs(H, W, 1 / wl.T, 1 / H, m0), tol=1e-10, m=40, maxit=1000)
    assert np.array_equal(r.x, ms[0])


def test_exact_galerkin_projection_pins(orc):
    # G = V^T A_i V: the residual of x0 is orthogonal to the basis (Galerkin
    # condition), and with the seed's own operator it equals the paper's
    # projection through H_a
    from paper_2511_17634_gb300 import synth
    wl = synth.config(2, T=1000, ntargets=4)
    g = wl.groups[0]
    H, W, N = g.H, g.W, g.N
    dt, h, g2 = 1.0 / wl.T, 1.0 / H, float(wl.g2[300])
    ms = g.seeds.reshape(len(g.seeds), -1)[0]
    mt = g.targets.reshape(len(g.targets), -1)[1]
    Cs = orc.coeffs(H, W, g2, dt, h, ms)
    r = orc.gmres(H, W, Cs, orc.rhs(H, W, dt, h, ms), tol=1e-10, m=40, maxit=400, capture=40)
    Ct = orc.coeffs(H, W, g2, dt, h, mt)
    b = orc.rhs(H, W, dt, h, mt)
    x0, sing = orc.project_galerkin(H, W, Ct, r.V, r.a, b)
    assert not sing
    res = b - orc.apply(H, W, Ct, x0)
    assert np.abs(r.V[:r.a] @ res).max() <= 1e-11 * np.linalg.norm(b)
    xs, _ = orc.project_galerkin(H, W, Cs, r.V, r.a, b)
    xp, _ = orc.project(r.V, r.Hbar, r.a, r.has_next, b)
    assert np.abs(xs - xp).max() <= 1e-10 * np.abs(xp).max()
    # residual form: x1 = xi + V G^-1 V^T (b - A xi) also satisfies the
    # Galerkin condition, and equals x0 when xi lies in span(V)
    xi = np.linspace(0, 1, N)
    x1, _ = orc.project_galerkin(H, W, Ct, r.V, r.a, b - orc.apply(H, W, Ct, xi), xinit=xi)
    assert np.abs(r.V[:r.a] @ (b - orc.apply(H, W, Ct, x1))).max() <= 1e-11 * np.linalg.norm(b)
    xv = r.V[:r.a].T @ np.random.default_rng(1).normal(size=r.a)
    x2, _ = orc.project_galerkin(H, W, Ct, r.V, r.a, b - orc.apply(H, W, Ct, xv), xinit=xv)
    assert np.abs(x2 - x0).max() <= 1e-9 * np.abs(x0).max()


def test_picard_iterations_pins(orc):
    # K = 1 is the one-solve step; more Picard iterations converge to the
    # fixed point A(m^n) m^n = m^{n-1}/dt of the implicit step; with g = 0 the
    # operator does not depend on m~ and extra iterations change nothing
    H, W = 9, 7
    N = H * W
    rng = np.random.default_rng(4)
    m0 = rng.uniform(0, 1, (2, N))
    dt, h, g2 = 0.02, 1.0 / H, 0.4
    kw = dict(mode=1, tol_seed=1e-13, m_seed=40, a=40, tol_ref=1e-13, m_ref=40)
    ref = m0.copy(); s1 = m0[:1].copy()
    orc.march_step(H, W, dt, h, g2, s1, ref, [0, 0], **kw)
    one = m0.copy(); s2 = m0[:1].copy()
    orc.march_step(H, W, dt, h, g2, s2, one, [0, 0], picard=1, **kw)
    assert np.array_equal(one, ref)
    res = []
    for K in (1, 2, 4, 8):
        x = m0.copy(); s = m0[:1].copy()
        orc.march_step(H, W, dt, h, g2, s, x, [0, 0], picard=K, **kw)
        C = orc.coeffs(H, W, g2, dt, h, x[0])          # A(m^n) from the result itself
        r = orc.apply(H, W, C, x[0]) - orc.rhs(H, W, dt, h, m0[0])
        res.append(np.linalg.norm(r) / np.linalg.norm(m0[0] / dt))
    assert res[1] < 0.2 * res[0] and res[3] < 1e-10
    x0 = m0.copy(); xs = m0[:1].copy()
    orc.march_step(H, W, dt, h, 0.0, xs, x0, [0, 0], **kw)
    x3 = m0.copy(); xs3 = m0[:1].copy()
    orc.march_step(H, W, dt, h, 0.0, xs3, x3, [0, 0], picard=3, **kw)
    assert np.allclose(x3, x0, rtol=1e-12, atol=0)


@pytest.mark.parametrize("H,W", [(3, 3), (4, 5), (8, 8)])
def test_bicgstab_matches_dense_solve(orc, H, W):
    # Sec. 3, Phase 1 as printed: BiCGSTAB reaches the solution of the
    # nonsymmetric five-point system (drift f != 0) that a dense solve gives
    rng = np.random.default_rng(40 + H * W)
    dt, h, g2 = 0.01, 1 / H, 0.25
    C = orc.coeffs(H, W, g2, dt, h, rng.uniform(0, 1, H * W), rng.normal(size=H * W),
                   rng.normal(size=H * W))
    A = np.stack([orc.apply(H, W, C, e) for e in np.eye(H * W)], axis=1)
    assert np.abs(A - A.T).max() > 1e-3 * np.abs(A).max()          # really nonsymmetric
    b = rng.normal(size=H * W)
    x_np = np.linalg.solve(A, b)
    r = orc.bicgstab(H, W, C, b, tol=1e-13, maxit=500)
    assert r.status == 0 and r.iters <= 2 * H * W
    assert np.linalg.norm(r.x - x_np) <= 1e-11 * np.linalg.norm(x_np)
    assert abs(np.linalg.norm(b - A @ r.x) / np.linalg.norm(b) - r.rel_res) <= 1e-14


@pytest.mark.parametrize("H,W", [(2, 3), (3, 3), (4, 5), (8, 8)])
def test_bicgstab_finite_termination(orc, H, W):
    # like BiCG, BiCGSTAB ends in at most N iterations in exact arithmetic (no
    # breakdown); on strongly convective systems (large drift, dt = 1, far
    # from the identity) rounding costs it a few more, never hundreds
    rng = np.random.default_rng(40 + H * W)
    N = H * W
    b = rng.normal(size=N)
    for dt in (1.0, 100.0):
        C = orc.coeffs(H, W, 4.0, dt, 1 / H, rng.uniform(0, 1, N), 30 * rng.normal(size=N),
                       30 * rng.normal(size=N))
        r = orc.bicgstab(H, W, C, b, tol=1e-13, maxit=500)
        assert r.status == 0 and r.iters <= 1.5 * N + 2


def test_bicgstab_hard_system_and_restart(orc):
    # the worse-conditioned g = 0.5 system needs many iterations; with a
    # small iteration cap it stops short and reports it, and resuming from
    # the returned iterate finishes the solve
    H = W = 16
    C, b, A = _hard_system(orc)
    r = orc.bicgstab(H, W, C, b, tol=1e-12, maxit=400)
    assert r.status == 0 and r.rel_res <= 1e-12
    assert np.linalg.norm(r.x - np.linalg.solve(A, b)) <= 1e-10 * np.linalg.norm(r.x)
    part = orc.bicgstab(H, W, C, b, tol=1e-12, maxit=2)
    assert part.status == orc.NOT_CONVERGED and part.iters == 2
    rest = orc.bicgstab(H, W, C, b, x0=part.x, tol=1e-12, maxit=400)
    assert rest.status == 0 and np.linalg.norm(rest.x - r.x) <= 1e-10 * np.linalg.norm(r.x)


def test_bicgstab_key_vectors_span_the_krylov_spaces(orc):
    # the j-th kept vector (r_0, s_1, r_1, s_2, ...) lies in K_{j+1}(A, r_0):
    # the first j kept vectors span the same space as the first j Arnoldi
    # vectors of GMRES from the same start (x0 = 0, r_0 = b)
    H = W = 16
    C, b, A = _hard_system(orc)
    rb = orc.bicgstab(H, W, C, b, tol=1e-12, maxit=400, capture=8)
    rg = orc.gmres(H, W, C, b, tol=1e-13, m=40, maxit=400, capture=8)
    Vb, Vg = rb.V.T, rg.V.T
    assert Vb.shape[1] == 8
    assert np.abs(Vb.T @ Vb - np.eye(8)).max() <= 1e-12
    assert np.allclose(Vb[:, 0], b / np.linalg.norm(b), rtol=0, atol=1e-15)
    for j in range(1, 8):
        Q = Vg[:, :j]
        assert np.linalg.norm(Vb[:, :j] - Q @ (Q.T @ Vb[:, :j])) <= 1e-12
        assert np.linalg.norm(Vb[:, j] - Q @ (Q.T @ Vb[:, j])) >= 0.5     # and grows


def test_dense_projection_pins(orc):
    # x0 = V (V^T A V)^{-1} V^T b depends only on span(V): on the BiCGSTAB
    # basis (explicit A_proj) it equals the paper's Hessenberg projection on
    # the GMRES basis of the same Krylov space, satisfies the Galerkin
    # condition, and reaches the exact solution on a full basis
    H = W = 16
    C, b, A = _hard_system(orc)
    for a in (2, 4):
        rb = orc.bicgstab(H, W, C, b, tol=1e-12, maxit=400, capture=a)
        rg = orc.gmres(H, W, C, b, tol=1e-13, m=40, maxit=400, capture=a)
        V = rb.V
        Ap = V @ A @ V.T
        xd, sing = orc.project_dense(V, Ap, b)
        assert not sing
        xh, _ = orc.project(rg.V, rg.Hbar, rg.a, rg.has_next, b)
        assert np.linalg.norm(xd - xh) <= 1e-12 * np.linalg.norm(xh)
        assert np.abs(V @ (b - A @ xd)).max() <= 1e-11 * np.linalg.norm(b)
        # a transposed A_proj is a different (wrong) projection
        xt, _ = orc.project_dense(V, Ap.T, b)
        assert np.linalg.norm(xt - xh) >= 1e-3 * np.linalg.norm(xh)
    Hs, Ws = 3, 3
    rng = np.random.default_rng(12)
    Cs = orc.coeffs(Hs, Ws, 0.25, 0.01, 1 / 3, rng.uniform(0, 1, 9), rng.normal(size=9),
                    rng.normal(size=9))
    As = np.stack([orc.apply(Hs, Ws, Cs, e) for e in np.eye(9)], axis=1)
    Q, _ = np.linalg.qr(rng.normal(size=(9, 9)))
    bs = rng.normal(size=9)
    x9, _ = orc.project_dense(Q.T, Q.T @ As @ Q, bs, xinit=np.zeros(9))
    assert np.linalg.norm(x9 - np.linalg.solve(As, bs)) <= 1e-12 * np.linalg.norm(x9)


def test_march_bicgstab_seeds(orc):
    # the march with the paper's BiCGSTAB seeds reaches the same trajectory as
    # with GMRES seeds (both refine to 1e-12), the seed states too, and the
    # projected guesses are as good (targets need as many refine steps)
    wl = synth.config(1, T=8)
    g = wl.groups[0]
    kw = dict(m_seed=30, a=30, m_ref=30, tol_ref=1e-12, tol_seed=1e-12)
    msg, mtg, stg = orc.march(g.H, g.W, wl.T, wl.g2, g.seeds, g.targets, g.target_seed, **kw)
    msb, mtb, stb = orc.march(g.H, g.W, wl.T, wl.g2, g.seeds, g.targets, g.target_seed,
                              seed_solver=orc.SEED_BICGSTAB, **kw)
    assert all((s.tgt_status == 0).all() for s in stb)
    assert np.abs(mtb - mtg).max() <= 1e-9 * np.abs(mtg).max()
    assert np.abs(msb - msg).max() <= 1e-9 * np.abs(msg).max()
    x0b = np.concatenate([s.tgt_x0res for s in stb])
    x0g = np.concatenate([s.tgt_x0res for s in stg])
    assert np.all(x0b < 1) and np.median(x0b) <= 10 * np.median(x0g)
    # the first step's guesses are x0 = V (V^T A_seed V)^{-1} V^T b_i with the
    # seed's BiCGSTAB key vectors, A_proj formed from the dense operator here
    H, W, N = g.H, g.W, g.N
    dt, h = 1.0 / wl.T, 1.0 / H
    m0 = g.seeds.reshape(len(g.seeds), -1)
    tg = g.targets.reshape(len(g.targets), -1)
    for t in range(len(tg)):
        s0 = m0[g.target_seed[t]]
        Cs = orc.coeffs(H, W, wl.g2[0], dt, h, s0)
        As = np.stack([orc.apply(H, W, Cs, e) for e in np.eye(N)], axis=1)
        V = orc.bicgstab(H, W, Cs, orc.rhs(H, W, dt, h, s0), tol=1e-12, maxit=1000, capture=30).V
        bt = orc.rhs(H, W, dt, h, tg[t])
        x0, _ = orc.project_dense(V, V @ As @ V.T, bt)
        Ct = orc.coeffs(H, W, wl.g2[0], dt, h, tg[t])
        res = np.linalg.norm(bt - orc.apply(H, W, Ct, x0)) / np.linalg.norm(bt)
        assert abs(res - stb[0].tgt_x0res[t]) <= 1e-9 * res


def _span_gap(A, B):
    # largest distance of a column of B from span(A) (A: orthonormal columns)
    return np.linalg.norm(B - A @ (A.T @ B), axis=0).max()


def test_accumulate_pins(orc):
    # seed cycling (Sec. 5.2): the new seed's space first and whole, older
    # vectors fill the rest up to the cap, nothing dependent is kept
    H = W = 16
    N = H * W
    C, b, A = _hard_system(orc)
    rng = np.random.default_rng(21)
    Q, _ = np.linalg.qr(rng.normal(size=(N, 12)))
    Vown, Vprev = Q[:, :5].T, Q[:, 5:12].T            # rows, independent spaces
    V, Ap = orc.accumulate(H, W, C, Vown, Vprev, 40)
    assert V.shape[0] == 12
    assert np.abs(V @ V.T - np.eye(12)).max() <= 1e-13
    assert _span_gap(V[:5].T, Vown.T) <= 1e-13                  # own space first
    assert _span_gap(V.T, Q) <= 1e-13                            # everything kept
    assert np.abs(Ap - V @ A @ V.T).max() <= 1e-12 * np.abs(A).max()
    # a cap below the total keeps the own space and the first older vectors
    Vc, _ = orc.accumulate(H, W, C, Vown, Vprev, 8)
    assert Vc.shape[0] == 8 and _span_gap(Vc[:5].T, Vown.T) <= 1e-13
    assert _span_gap(Vc.T, Vprev[:3].T) <= 1e-12
    # the same space again adds nothing; a mixed one adds only what is new
    Vs, _ = orc.accumulate(H, W, C, Vown, Vown[::-1] * 2.0, 40)
    assert Vs.shape[0] == 5
    Vm, _ = orc.accumulate(H, W, C, Vown, np.vstack([Vown[1] + Vown[2], Vprev[0]]), 40)
    assert Vm.shape[0] == 6 and _span_gap(Vm.T, Vprev[:1].T) <= 1e-13
    # Galerkin condition with the seed's operator, for the seed's own rhs
    x0, sing = orc.project_dense(V, Ap, b)
    assert not sing and np.abs(V @ (b - A @ x0)).max() <= 1e-11 * np.linalg.norm(b)


def test_march_seed_cycling(orc):
    # a chain of three seeds (0 <- 1 <- 2): the guesses of the targets of seed
    # 2 come from the span of all three seeds' GMRES bases with seed 2's
    # operator; the trajectory is the plain march's (all refined to 1e-12)
    wl = synth.config(2, T=1000, ntargets=6)
    g = wl.groups[0]
    H, W, N = g.H, g.W, g.N
    seeds = g.seeds.reshape(len(g.seeds), -1)[[0, 3, 6]]        # three channels 0 of three templates
    tg = g.targets.reshape(len(g.targets), -1)[:6]
    ts = np.array([0, 1, 2, 2, 1, 0], dtype=np.int32)
    prev = np.array([-1, 0, 1], dtype=np.int32)
    n = 400
    dt, h, g2 = 1.0 / wl.T, 1.0 / H, float(wl.g2[n])
    kw = dict(mode=0, tol_seed=1e-10, m_seed=40, a=40, tol_ref=1e-12, m_ref=40)
    ms, mt = seeds.copy(), tg.copy()
    st = orc.march_step(H, W, dt, h, g2, ms, mt, ts, seed_prev=prev, **kw)
    ms0, mt0 = seeds.copy(), tg.copy()
    orc.march_step(H, W, dt, h, g2, ms0, mt0, ts, mode=1, tol_seed=1e-10, m_seed=40, a=40,
                   tol_ref=1e-12, m_ref=40)
    assert np.abs(mt - mt0).max() <= 1e-9 * np.abs(mt0).max()
    assert np.array_equal(ms, ms0)                              # seeds are solved as before
    bases = []
    for s in range(3):
        Cs = orc.coeffs(H, W, g2, dt, h, seeds[s])
        r = orc.gmres(H, W, Cs, orc.rhs(H, W, dt, h, seeds[s]), tol=1e-10, m=40, maxit=1000,
                      capture=40)
        bases.append(r.V[:r.a])
    C2 = orc.coeffs(H, W, g2, dt, h, seeds[2])
    A2 = np.stack([orc.apply(H, W, C2, e) for e in np.eye(N)], axis=1)
    Q, _ = np.linalg.qr(np.vstack(bases).T)                      # any orthonormal basis of the span
    for t in (2, 3):
        bt = orc.rhs(H, W, dt, h, tg[t])
        x0, _ = orc.project_dense(Q.T, Q.T @ A2 @ Q, bt)
        Ct = orc.coeffs(H, W, g2, dt, h, tg[t])
        res = np.linalg.norm(bt - orc.apply(H, W, Ct, x0)) / np.linalg.norm(bt)
        assert abs(res - st.tgt_x0res[t]) <= 1e-12 * res
    assert sum(b.shape[0] for b in bases) <= 40
