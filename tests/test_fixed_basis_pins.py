"""Pins of the oracle's fixed basis dimension (Sec. 3: the stored V_a^n spans
the a-dimensional Krylov space K_a(A^n, r0); Sec. 5.2 runs a = 20).

With ``fixed=True`` the seed's first GMRES cycle keeps taking Arnoldi steps
after its residual test is met, until it has a = min(cap_a, m) vectors (an
exact breakdown or maxit end it earlier).  What pins it, other than the
oracle itself:

* the Arnoldi identities and orthonormality hold for all a + 1 vectors, and
  the first a' columns equal the converged-cycle capture bit for bit (the
  arithmetic up to step a' is the same);
* the cycle's iterate is the GMRES minimiser over K_a (a stale iterate from
  step a' would leave its larger residual);
* the projection of the seed's own right-hand side onto the fixed basis is
  the FOM iterate at step a (Saad 2003, Prop. 6.7) and meets the Galerkin
  condition;
* on a grid whose operator has three distinct eigenvalues the Krylov space
  stops growing at dimension 3: the basis ends at the exact breakdown.
"""
import numpy as np
import pytest

from paper_2511_17634_gb300 import synth


def _seed_system(orc, n=999):
    # the tiny workload's seed at its last timestep (largest g^2): converges
    # in a handful of steps at 1e-10, well short of a = 20
    wl = synth.config(1)
    g = wl.groups[0]
    H, W, T = g.H, g.W, wl.T
    mt = np.ascontiguousarray(g.seeds[0]).reshape(-1)
    C = orc.coeffs(H, W, wl.g2[min(n, T - 1)], 1 / T, 1 / H, mt)
    b = orc.rhs(H, W, 1 / T, 1 / H, mt)
    A = np.stack([orc.apply(H, W, C, e) for e in np.eye(H * W)], axis=1)
    return H, W, C, b, A


def test_fixed_basis_keeps_a_vectors_with_arnoldi_identities(orc):
    H, W, C, b, A = _seed_system(orc)
    a = 20
    conv = orc.gmres(H, W, C, b, tol=1e-10, m=40, maxit=400, capture=a)
    assert conv.status == 0 and conv.a < a          # the converged cycle is shorter
    r = orc.gmres(H, W, C, b, tol=1e-10, m=40, maxit=400, capture=a, fixed=True)
    assert r.status == 0 and r.a == a and r.has_next == 1 and r.iters == a
    V = r.V.T
    assert np.abs(V.T @ V - np.eye(a + 1)).max() <= 1e-13
    normA = np.linalg.norm(A, 2)
    assert np.linalg.norm(A @ V[:, :a] - V @ r.Hbar) <= 1e-13 * normA
    assert np.abs(V[:, :a].T @ A @ V[:, :a] - r.Hbar[:a]).max() <= 1e-12 * normA
    # the first a' steps are the converged capture, bit for bit
    ap = conv.a
    assert np.array_equal(r.V[:ap + conv.has_next], conv.V)
    assert np.array_equal(r.Hbar[:ap + 1, :ap], conv.Hbar)


def test_fixed_basis_iterate_is_the_gmres_minimiser_over_k_a(orc):
    H, W, C, b, A = _seed_system(orc)
    a = 20
    conv = orc.gmres(H, W, C, b, tol=1e-10, m=40, maxit=400, capture=a)
    r = orc.gmres(H, W, C, b, tol=1e-10, m=40, maxit=400, capture=a, fixed=True)
    Va = r.V[:a].T
    y, *_ = np.linalg.lstsq(A @ Va, b, rcond=None)
    xmin = Va @ y
    assert np.linalg.norm(r.x - xmin) <= 1e-12 * np.linalg.norm(xmin)
    true = np.linalg.norm(b - A @ r.x) / np.linalg.norm(b)
    assert abs(true - r.rel_res) <= 1e-14
    # far below the test's 1e-10 and below the converged cycle's residual
    assert r.rel_res <= 1e-13 < conv.rel_res


def test_projection_onto_fixed_basis_is_fom_iterate_at_step_a(orc):
    # a loose tolerance ends the converged cycle after ~3 steps; the fixed
    # basis of a = 6 then still leaves a residual well above rounding, so
    # the FOM residual formula can be checked to a tight relative bound
    H, W, C, b, A = _seed_system(orc)
    a = 6
    conv = orc.gmres(H, W, C, b, tol=1e-3, m=40, maxit=400, capture=a)
    assert conv.a < a
    r = orc.gmres(H, W, C, b, tol=1e-3, m=40, maxit=400, capture=a, fixed=True)
    assert r.a == a and r.has_next == 1
    x0, lsq = orc.project(r.V, r.Hbar, r.a, r.has_next, b)
    assert not lsq
    alpha = np.linalg.solve(r.Hbar[:a], r.V[:a] @ b)
    res = b - A @ x0
    expect = r.Hbar[a, a - 1] * abs(alpha[-1])
    assert expect > 1e-9 * np.linalg.norm(b)
    assert abs(np.linalg.norm(res) - expect) <= 1e-6 * expect
    assert abs(res @ r.V[a]) / np.linalg.norm(res) >= 1 - 1e-8
    assert np.abs(r.V[:a] @ res).max() <= 1e-12 * np.linalg.norm(b)
    # more basis vectors, smaller FOM residual than the converged capture's
    x0c, _ = orc.project(conv.V, conv.Hbar, conv.a, conv.has_next, b)
    assert np.linalg.norm(res) < np.linalg.norm(b - A @ x0c)


def test_fixed_basis_ends_at_exact_breakdown(orc):
    # 2x2 grid, m~ = 0, f = 0: A = I/dt + c (Dirichlet Laplacian) has the
    # eigenvalues 1/dt + c {2, 4, 4, 6}, so a generic b spans a Krylov space
    # of dimension 3 and Arnoldi breaks down at step 3 whatever a asks
    H = W = 2
    C = orc.coeffs(H, W, 0.5, 0.01, 0.5, np.zeros(4))
    A = np.stack([orc.apply(H, W, C, e) for e in np.eye(4)], axis=1)
    assert len(np.unique(np.round(np.linalg.eigvalsh(A), 9))) == 3
    b = np.array([1.0, 0.3, -0.7, 2.0])
    r = orc.gmres(H, W, C, b, tol=1e-10, m=10, maxit=100, capture=10, fixed=True)
    assert r.status == 0 and r.a == 3 and r.has_next == 0
    assert np.all(np.isfinite(r.V)) and np.abs(r.V @ r.V.T - np.eye(3)).max() <= 1e-14
    assert np.linalg.norm(r.x - np.linalg.solve(A, b)) <= 1e-13 * np.linalg.norm(r.x)


@pytest.mark.parametrize("fixed", [False, True])
def test_march_with_fixed_basis_reaches_the_plain_trajectory(orc, fixed):
    wl = synth.config(1, T=6)
    g = wl.groups[0]
    kw = dict(m_seed=30, a=20, m_ref=30, tol_ref=1e-12)
    _, ref, _ = orc.march(g.H, g.W, wl.T, wl.g2, g.seeds, g.targets, g.target_seed,
                          mode=orc.MODE_PLAIN, **kw)
    ms, mt, st = orc.march(g.H, g.W, wl.T, wl.g2, g.seeds, g.targets, g.target_seed,
                           mode=orc.MODE_PROJECTED, fixed_a=fixed, **kw)
    assert all((s.tgt_status == 0).all() for s in st)
    assert np.abs(mt - ref).max() <= 1e-9 * np.abs(ref).max()
    if fixed:
        # every seed solve took at least a steps (its first cycle; these
        # short-T systems need more than 20 at tol 1e-10 from step 3 on)
        assert all((s.seed_iters >= 20).all() for s in st)


def test_march_seed_update_with_fixed_basis_equals_fixed_gmres(orc):
    wl = synth.config(1, T=4)
    g = wl.groups[0]
    H, W = g.H, g.W
    ms = g.seeds.reshape(1, -1).copy()
    mt = g.targets.reshape(len(g.targets), -1).copy()
    m0 = ms[0].copy()
    orc.march_step(H, W, 1 / wl.T, 1 / H, wl.g2[0], ms, mt, g.target_seed, a=20, fixed_a=True)
    C = orc.coeffs(H, W, wl.g2[0], 1 / wl.T, 1 / H, m0)
    r = orc.gmres(H, W, C, orc.rhs(H, W, 1 / wl.T, 1 / H, m0), tol=1e-10, m=40, maxit=1000,
                  capture=20, fixed=True)
    assert np.array_equal(r.x, ms[0])
