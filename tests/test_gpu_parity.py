"""GPU parity of every step of the hot path against the FP64 CPU oracle,
through the C ABI (include/kp.h) via the thin binding.

Tolerances.  Both sides solve to a relative residual `tol`; the systems have
cond_inf(A) <= 1 + 8 c dt (M-matrix bound, at most ~2.3 on the workloads), so
each solution is within ~cond*tol of the exact one and the two within twice
that.  The operator itself is compared to 1e-13 relative (a handful of FP64
roundings in a different order).  The spec bar is 1e-6 relative.
"""
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


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("H,W", [(5, 3), (28, 28), (32, 32), (17, 40), (64, 64), (1, 1)])
def test_apply_and_rhs_match_oracle(kp, orc, H, W):
    rng = np.random.default_rng(H * 100 + W)
    n = 3
    N = H * W
    mt, x, fx, fy = (rng.normal(size=(n, N)) for _ in range(4))
    g2 = rng.uniform(0.01, 0.5, n)
    ctx = kp.Context(max_n=max(N, 16))
    ops = kp.make_ops(H, W, 0.01, g2, 1.0 / H, _dev(mt), _dev(fx), _dev(fy))
    y = torch.zeros((n, N), dtype=torch.float64, device="cuda")
    dx = _dev(x)
    ctx.apply(ops, dx, y)
    b = torch.zeros_like(y)
    ctx.rhs(ops, dx, b)
    torch.cuda.synchronize()
    for k in range(n):
        C = orc.coeffs(H, W, g2[k], 0.01, 1.0 / H, mt[k], fx[k], fy[k])
        assert _rel(y[k].cpu().numpy(), orc.apply(H, W, C, x[k])) <= 1e-13
        assert _rel(b[k].cpu().numpy(), orc.rhs(H, W, 0.01, 1.0 / H, x[k], fx[k], fy[k])) <= 1e-14


def _seed_systems(wl, n_step):
    g = wl.groups[0]
    H, W = g.H, g.W
    ms = g.seeds.reshape(len(g.seeds), -1)
    return H, W, 1.0 / wl.T, 1.0 / H, float(wl.g2[n_step]), ms


@pytest.mark.parametrize("reorth", [0, 1])
@pytest.mark.parametrize("smem_vectors", [0, 3])
def test_seed_solve_and_basis_match_oracle(kp, orc, reorth, smem_vectors):
    wl = synth.config(2, T=1000, ntargets=4)
    H, W, dt, h, g2, ms = _seed_systems(wl, 999)
    ns, N = ms.shape
    ctx = kp.Context(max_a=40, max_n=N, reorth=reorth, smem_vectors=smem_vectors)
    mt = _dev(ms)
    ops = kp.make_ops(H, W, dt, g2, h, mt)
    b = torch.zeros_like(mt)
    ctx.rhs(ops, mt, b)
    x = torch.zeros_like(mt)
    info = ctx.seed_solve(ops, b, x, tol=1e-10, m=40, maxit=400)
    for s in range(ns):
        ctx.store_basis(s, 7, s)
    torch.cuda.synchronize()
    iters, status, res = kp.decode_info(info)
    assert (status == 0).all() and (res <= 1e-10).all()
    for s in range(ns):
        C = orc.coeffs(H, W, g2, dt, h, ms[s])
        r = orc.gmres(H, W, C, orc.rhs(H, W, dt, h, ms[s]), tol=1e-10, m=40, maxit=400, capture=40)
        assert abs(int(iters[s]) - r.iters) <= 1
        assert _rel(x[s].cpu().numpy(), r.x) <= 1e-9
        # true residual of the GPU answer, recomputed by the oracle
        xr = x[s].cpu().numpy()
        bb = orc.rhs(H, W, dt, h, ms[s])
        assert np.linalg.norm(bb - orc.apply(H, W, C, xr)) <= 1.01e-10 * np.linalg.norm(bb)
        a, hn, V, Hbar = ctx.basis_get(s, 7, N)
        if a == r.a:
            k = min(a, 6)   # leading Arnoldi vectors are well determined
            assert np.abs(V[:k].cpu().numpy() - r.V[:k]).max() <= 1e-9
            assert np.abs(Hbar[:k + 1, :k] - r.Hbar[:k + 1, :k]).max() <= 1e-9 * np.abs(r.Hbar).max()
        Vn = V.cpu().numpy()
        assert np.abs(Vn @ Vn.T - np.eye(Vn.shape[0])).max() <= 1e-12


@pytest.mark.parametrize("shape", [(0, 0), (128, 2), (128, 3), (128, 4), (64, 4), (256, 3)])
def test_projection_and_refine_match_oracle(kp, orc, shape):
    # every compiled one-block solver shape (threads per system, blocks per SM)
    wl = synth.config(2, T=1000, ntargets=24)
    g = wl.groups[0]
    H, W, N = g.H, g.W, g.N
    n = 500
    dt, h, g2 = 1.0 / wl.T, 1.0 / H, float(wl.g2[n])
    ms = g.seeds.reshape(len(g.seeds), -1)
    mt = g.targets.reshape(len(g.targets), -1)
    ctx = kp.Context(max_a=40, max_n=N, max_seeds=len(ms), block_threads=shape[0],
                     blocks_per_sm=shape[1])
    sm = _dev(ms)
    sops = kp.make_ops(H, W, dt, g2, h, sm)
    sb = torch.zeros_like(sm)
    ctx.rhs(sops, sm, sb)
    sx = torch.zeros_like(sm)
    ctx.seed_solve(sops, sb, sx, tol=1e-10, m=40, maxit=400)
    for s in range(len(ms)):
        ctx.store_basis(s, n, s)
    tm = _dev(mt)
    tops = kp.make_ops(H, W, dt, g2, h, tm)
    tb = torch.zeros_like(tm)
    ctx.rhs(tops, tm, tb)
    x0 = torch.zeros_like(tm)
    ctx.project_targets_multi(n, g.target_seed, tops, tb, x0)
    torch.cuda.synchronize()
    x0h = x0.cpu().numpy()
    xr = x0.clone()
    info = ctx.refine(tops, tb, xr, tol=1e-10, m=40, maxit=400)
    torch.cuda.synchronize()
    iters, status, res = kp.decode_info(info)
    assert (status == 0).all()
    bases = {}
    for s in range(len(ms)):
        C = orc.coeffs(H, W, g2, dt, h, ms[s])
        bases[s] = orc.gmres(H, W, C, orc.rhs(H, W, dt, h, ms[s]), tol=1e-10, m=40, maxit=400,
                             capture=40)
    for t in range(len(mt)):
        r = bases[int(g.target_seed[t])]
        b = orc.rhs(H, W, dt, h, mt[t])
        ox0, _ = orc.project(r.V, r.Hbar, r.a, r.has_next, b)
        assert _rel(x0h[t], ox0) <= 1e-9
        C = orc.coeffs(H, W, g2, dt, h, mt[t])
        ref = orc.gmres(H, W, C, b, x0=ox0, tol=1e-10, m=40, maxit=400)
        assert abs(int(iters[t]) - ref.iters) <= 1
        assert _rel(xr[t].cpu().numpy(), ref.x) <= 1e-9


def _gpu_march_step(kp, ctx, wl, gi, n, ms, mt, mode, tol_ref):
    g = wl.groups[gi]
    H, W = g.H, g.W
    dt, h, g2 = 1.0 / wl.T, 1.0 / H, float(wl.g2[n])
    sops = kp.make_ops(H, W, dt, g2, h, ms)
    sb = torch.zeros_like(ms)
    ctx.rhs(sops, ms, sb)
    sx = torch.zeros_like(ms)
    sinfo = ctx.seed_solve(sops, sb, sx, tol=wl.tol_seed, m=wl.m_seed, maxit=1000)
    for s in range(ms.shape[0]):
        ctx.store_basis(s, n, s)
    tops = kp.make_ops(H, W, dt, g2, h, mt)
    tb = torch.zeros_like(mt)
    ctx.rhs(tops, mt, tb)
    if mode == 0:
        x = torch.zeros_like(mt)
        ctx.project_targets_multi(n, g.target_seed, tops, tb, x)
    elif mode == 1:
        x = torch.zeros_like(mt)
    else:
        x = mt.clone()
    tinfo = ctx.refine(tops, tb, x, tol=tol_ref, m=wl.m, maxit=1000)
    ms.copy_(sx)
    mt.copy_(x)
    return sinfo, tinfo


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_march_step_parity(kp, orc, mode):
    # per step: the same m^{n-1} on both sides, tol 1e-10
    wl = synth.config(1)
    g = wl.groups[0]
    rng = np.random.default_rng(5)
    ms = g.seeds.reshape(1, -1).copy()
    mt = g.targets.reshape(len(g.targets), -1).copy()
    ctx = kp.Context(max_a=wl.a, max_n=g.N, max_seeds=4)
    for n in [0, 17, 49]:
        dms, dmt = _dev(ms), _dev(mt)
        si, ti = _gpu_march_step(kp, ctx, wl, 0, n, dms, dmt, mode, 1e-10)
        oms, omt = ms.copy(), mt.copy()
        st = orc.march_step(g.H, g.W, 1 / wl.T, 1 / g.H, float(wl.g2[n]), oms, omt, g.target_seed,
                            mode=mode, tol_seed=1e-10, m_seed=wl.m_seed, a=wl.a, tol_ref=1e-10,
                            m_ref=wl.m)
        torch.cuda.synchronize()
        assert np.abs(dms.cpu().numpy() - oms).max() <= 1e-8 * np.abs(oms).max()
        assert np.abs(dmt.cpu().numpy() - omt).max() <= 1e-8 * np.abs(omt).max()
        it, stt, res = kp.decode_info(ti)
        assert (stt == 0).all() and (res <= 1e-10).all()
        assert (np.abs(it - st.tgt_iters) <= 1).all()
        ms = ms + 0.01 * rng.normal(size=ms.shape)      # move to a different m^{n-1}
        mt = mt + 0.01 * rng.normal(size=mt.shape)


def test_trajectory_parity_tiny(kp, orc):
    # whole trajectory of the tiny workload (28x28x1, 1 seed + 4 targets, T=50)
    # at tol 1e-12 on both sides
    wl = synth.config(1)
    g = wl.groups[0]
    ctx = kp.Context(max_a=wl.a, max_n=g.N, max_seeds=4)
    dms = _dev(g.seeds.reshape(1, -1))
    dmt = _dev(g.targets.reshape(len(g.targets), -1))
    for n in range(wl.T):
        _gpu_march_step(kp, ctx, wl, 0, n, dms, dmt, 0, 1e-12)
    oms, omt, _ = orc.march(g.H, g.W, wl.T, wl.g2, g.seeds, g.targets, g.target_seed,
                            tol_seed=1e-10, m_seed=wl.m_seed, a=wl.a, tol_ref=1e-12, m_ref=wl.m)
    torch.cuda.synchronize()
    assert np.abs(dmt.cpu().numpy() - omt).max() <= 1e-6 * np.abs(omt).max()
    assert np.abs(dmt.cpu().numpy() - omt).max() <= 1e-9 * np.abs(omt).max()


def test_edge_cases(kp, orc):
    ctx = kp.Context(max_n=4096, max_seeds=4)
    H, W = 7, 5
    N = H * W
    rng = np.random.default_rng(3)
    mt = _dev(rng.uniform(0, 1, (3, N)))
    ops = kp.make_ops(H, W, 0.01, 0.3, 1 / H, mt)
    # empty batch
    e = torch.zeros((0, N), dtype=torch.float64, device="cuda")
    ctx.refine(kp.make_ops(H, W, 0.01, 0.3, 1 / H, e), e, e)
    # b = 0 -> x = 0, converged, 0 iterations
    b = torch.zeros((3, N), dtype=torch.float64, device="cuda")
    x = _dev(rng.normal(size=(3, N)))
    it, st, rr = kp.decode_info(ctx.refine(ops, b, x))
    assert (it == 0).all() and (st == 0).all() and float(x.abs().max()) == 0.0
    # maxit = 0: untouched guess, NOT_CONVERGED
    b = _dev(rng.normal(size=(3, N)))
    x = torch.zeros_like(b)
    it, st, rr = kp.decode_info(ctx.refine(ops, b, x, maxit=0))
    assert (st == kp.NOT_CONVERGED).all() and (it == 0).all() and float(x.abs().max()) == 0.0
    assert np.allclose(rr, 1.0)
    # NaN in b -> BREAKDOWN status, no hang
    bn = b.clone()
    bn[1, 3] = float("nan")
    x = torch.zeros_like(b)
    it, st, rr = kp.decode_info(ctx.refine(ops, bn, x, maxit=50))
    assert st[1] == kp.BREAKDOWN and st[0] == 0 and st[2] == 0
    # g2 = 0: A = I/dt, one iteration, x = dt b
    ops0 = kp.make_ops(H, W, 0.01, 0.0, 1 / H, mt)
    x = torch.zeros_like(b)
    it, st, rr = kp.decode_info(ctx.refine(ops0, b, x, tol=1e-12))
    assert (it == 1).all() and torch.allclose(x, 0.01 * b, rtol=1e-14, atol=0)
    # m = 1 (restart every step) still converges
    x = torch.zeros_like(b)
    it, st, rr = kp.decode_info(ctx.refine(ops, b, x, tol=1e-10, m=1, maxit=500))
    assert (st == 0).all() and (rr <= 1e-10).all()
    # largest grid this kernel family takes (64x64) and a 1x1 grid
    for (h_, w_) in [(64, 64), (1, 1), (3, 1)]:
        n_ = h_ * w_
        m_ = _dev(rng.uniform(0, 1, (2, n_)))
        o_ = kp.make_ops(h_, w_, 1e-3, 0.02, 1 / h_, m_)
        bb = _dev(rng.normal(size=(2, n_)))
        xx = torch.zeros_like(bb)
        it, st, rr = kp.decode_info(ctx.refine(o_, bb, xx, tol=1e-10))
        assert (st == 0).all()
        for k in range(2):
            C = orc.coeffs(h_, w_, 0.02, 1e-3, 1 / h_, m_[k].cpu().numpy())
            ref = orc.gmres(h_, w_, C, bb[k].cpu().numpy(), tol=1e-12, m=40, maxit=400)
            assert _rel(xx[k].cpu().numpy(), ref.x) <= 1e-9
    # argument errors are reported, not crashed on
    with pytest.raises(kp.KPError):
        ctx.refine(ops, b, x, m=0)
    with pytest.raises(kp.KPError):
        big = kp.make_ops(128, 128, 0.01, 0.3, 1 / 128, mt)   # N > max_n
        ctx.refine(big, b, x)
    with pytest.raises(kp.KPError) as ei:
        ctx.project_targets(0, 123, ops, b, x)                # nothing stored
    assert ei.value.status == kp.ERR_NO_BASIS
