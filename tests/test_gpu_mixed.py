"""Mixed precision (FP32 Krylov inside FP64 iterative refinement): every solve
still meets the FP64 true-residual tolerance, so its distance to the FP64
oracle is bounded by cond(A) * tol like the FP64 path's; the tests state the
measured max and median relative errors against the oracle."""
import numpy as np
import pytest

from paper_2511_17634_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_17634_gb300 import build
    build.build()
    from paper_2511_17634_gb300 import kp as K
    return K


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


@pytest.mark.parametrize("H,W,g2,dt", [(32, 32, 0.02, 1e-3), (64, 64, 0.02, 1e-3),
                                       (28, 28, 0.25, 1e-2), (7, 5, 0.3, 1e-2)])
def test_mixed_refine_meets_fp64_tolerance(kp, orc, H, W, g2, dt):
    rng = np.random.default_rng(H * W)
    N = H * W
    mt = rng.uniform(0, 1, (6, N))
    b = rng.normal(size=(6, N))
    ctx = kp.Context(max_n=max(N, 64), precision=kp.PREC_MIXED)
    dm, db = _dev(mt), _dev(b)
    ops = kp.make_ops(H, W, dt, g2, 1 / H, dm)
    x = torch.zeros_like(db)
    it, st, rr = kp.decode_info(ctx.refine(ops, db, x, tol=1e-10, m=30, maxit=500))
    torch.cuda.synchronize()
    assert (st == 0).all() and (rr <= 1e-10).all()
    for k in range(6):
        C = orc.coeffs(H, W, g2, dt, 1 / H, mt[k])
        xr = x[k].cpu().numpy()
        # FP64 true residual recomputed by the oracle
        assert np.linalg.norm(b[k] - orc.apply(H, W, C, xr)) <= 1.01e-10 * np.linalg.norm(b[k])
        ref = orc.gmres(H, W, C, b[k], tol=1e-13, m=40, maxit=800)
        assert np.linalg.norm(xr - ref.x) <= 1e-8 * np.linalg.norm(ref.x)


def test_mixed_seed_basis_and_projection(kp, orc):
    wl = synth.config(2, T=1000, ntargets=6)
    g = wl.groups[0]
    H, W, N = g.H, g.W, g.N
    n = 300
    dt, h, g2 = 1 / wl.T, 1 / H, float(wl.g2[n])
    ms = g.seeds.reshape(len(g.seeds), -1)
    mt = g.targets.reshape(len(g.targets), -1)
    ctx = kp.Context(max_seeds=len(ms), max_a=40, max_n=N, precision=kp.PREC_MIXED)
    sm_ = _dev(ms)
    sops = kp.make_ops(H, W, dt, g2, h, sm_)
    sb = torch.zeros_like(sm_)
    ctx.rhs(sops, sm_, sb)
    sx = torch.zeros_like(sm_)
    it, st, rr = kp.decode_info(ctx.seed_solve(sops, sb, sx, tol=1e-10, m=40, maxit=400))
    assert (st == 0).all() and (rr <= 1e-10).all()
    for s in range(len(ms)):
        ctx.store_basis(s, n, s)
    tm = _dev(mt)
    tops = kp.make_ops(H, W, dt, g2, h, tm)
    tb = torch.zeros_like(tm)
    ctx.rhs(tops, tm, tb)
    x0 = torch.zeros_like(tm)
    ctx.project_targets_multi(n, g.target_seed, tops, tb, x0)
    torch.cuda.synchronize()
    for t in range(len(mt)):
        s = int(g.target_seed[t])
        a, hn, V, Hb = ctx.basis_get(s, n, N)
        Vn = V.cpu().numpy()
        assert np.abs(Vn @ Vn.T - np.eye(Vn.shape[0])).max() <= 1e-5     # FP32 Arnoldi
        C = orc.coeffs(H, W, g2, dt, h, ms[s])
        ref = orc.gmres(H, W, C, orc.rhs(H, W, dt, h, ms[s]), tol=1e-10, m=40, maxit=400, capture=40)
        b = orc.rhs(H, W, dt, h, mt[t])
        ox0, _ = orc.project(ref.V, ref.Hbar, ref.a, ref.has_next, b)
        # initial guesses agree to FP32 accuracy of the basis
        assert np.linalg.norm(x0[t].cpu().numpy() - ox0) <= 1e-5 * np.linalg.norm(ox0)


def test_mixed_march_64x64_sampled_errors(kp, orc):
    # 64x64x3 blob workload (8 templates), first timesteps, all targets of a
    # small batch against the FP64 oracle: max and median relative error
    wl = synth.config(4, T=1000, ntargets=11)
    g = wl.groups[0]
    steps = 3
    ctx = kp.Context(max_seeds=2 * wl.n_seed_planes, max_a=wl.a, max_n=g.N,
                     precision=kp.PREC_MIXED)
    s_ = _dev(g.seeds.reshape(len(g.seeds), -1))
    t_ = _dev(g.targets.reshape(len(g.targets), -1))
    mr = kp.March(ctx, [(s_, t_, g.target_seed, g.H, g.W)], wl.T, wl.g2, mode=kp.MARCH_PROJECTED,
                  tol_seed=wl.tol_seed, tol=wl.tol, m_seed=wl.m_seed, m=wl.m)
    stats, _ = mr.run(0, steps, stats=True)
    torch.cuda.synchronize()
    assert all(s.not_converged == 0 and s.max_rel_res <= wl.tol for s in stats)
    oms, omt, _ = orc.march(g.H, g.W, wl.T, wl.g2, g.seeds, g.targets, g.target_seed, steps=steps,
                            tol_seed=wl.tol_seed, m_seed=wl.m_seed, a=wl.a, tol_ref=wl.tol,
                            m_ref=wl.m)
    gt = t_.cpu().numpy()
    rel = np.linalg.norm(gt - omt, axis=1) / np.linalg.norm(omt, axis=1)
    print(f"mixed vs FP64 oracle over {len(rel)} targets: max {rel.max():.2e} median {np.median(rel):.2e}")
    assert rel.max() <= 1e-6
