"""Grids above 4096 unknowns (up to 128x128 = 16384): the mixed-precision
solver on a thread-block cluster per system, against the FP64 oracle."""
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


@pytest.mark.parametrize("H,W", [(128, 128), (64, 128), (72, 64), (128, 40)])
def test_cluster_refine_meets_tolerance(kp, orc, H, W):
    rng = np.random.default_rng(H + W)
    N = H * W
    n = 3
    mt = rng.uniform(0, 1, (n, N))
    b = rng.normal(size=(n, N))
    ctx = kp.Context(max_n=16384, precision=kp.PREC_MIXED)
    dm, db = _dev(mt), _dev(b)
    ops = kp.make_ops(H, W, 1e-3, 0.02, 1 / H, dm)
    x = torch.zeros_like(db)
    it, st, rr = kp.decode_info(ctx.refine(ops, db, x, tol=1e-10, m=40, maxit=600))
    torch.cuda.synchronize()
    assert (st == 0).all() and (rr <= 1e-10).all(), (st, rr)
    for k in range(n):
        C = orc.coeffs(H, W, 0.02, 1e-3, 1 / H, mt[k])
        xr = x[k].cpu().numpy()
        assert np.linalg.norm(b[k] - orc.apply(H, W, C, xr)) <= 1.01e-10 * np.linalg.norm(b[k])
        ref = orc.gmres(H, W, C, b[k], tol=1e-13, m=40, maxit=800)
        assert np.linalg.norm(xr - ref.x) <= 1e-8 * np.linalg.norm(ref.x)


def test_cluster_march_128x128_sampled(kp, orc):
    wl = synth.config(5, T=1000, ntargets=3)
    g = wl.groups[0]
    steps = 2
    ctx = kp.Context(max_seeds=2 * wl.n_seed_planes, max_a=wl.a, max_n=g.N,
                     precision=kp.PREC_MIXED)
    s_ = _dev(g.seeds.reshape(len(g.seeds), -1))
    t_ = _dev(g.targets.reshape(len(g.targets), -1))
    mr = kp.March(ctx, [(s_, t_, g.target_seed, g.H, g.W)], wl.T, wl.g2, mode=kp.MARCH_PROJECTED,
                  tol_seed=wl.tol_seed, tol=wl.tol, m_seed=wl.m_seed, m=wl.m)
    stats, _ = mr.run(0, steps, stats=True)
    torch.cuda.synchronize()
    assert all(s.not_converged == 0 and s.max_rel_res <= wl.tol for s in stats)
    oms, omt, _ = orc.march(g.H, g.W, wl.T, wl.g2, g.seeds, g.targets, g.target_seed,
                            steps=steps, tol_seed=wl.tol_seed, m_seed=wl.m_seed, a=wl.a,
                            tol_ref=wl.tol, m_ref=wl.m)
    rel = np.linalg.norm(t_.cpu().numpy() - omt, axis=1) / np.linalg.norm(omt, axis=1)
    print(f"128x128 mixed vs FP64 oracle: max {rel.max():.2e} median {np.median(rel):.2e}")
    assert rel.max() <= 1e-6


@pytest.mark.parametrize("cs", [2, 4])
def test_cluster_forced_on_64x64(kp, orc, cs):
    # a 4096-point grid on a cluster of cs CTAs (kp_options.cluster_size)
    # instead of one 512-thread block: same tolerance against the oracle
    H = W = 64
    N = H * W
    rng = np.random.default_rng(cs)
    n = 3
    mt = rng.uniform(0, 1, (n, N))
    b = rng.normal(size=(n, N))
    ctx = kp.Context(max_n=N, precision=kp.PREC_MIXED, cluster_size=cs)
    dm, db = _dev(mt), _dev(b)
    ops = kp.make_ops(H, W, 1e-3, 0.02, 1 / H, dm)
    x = torch.zeros_like(db)
    it, st, rr = kp.decode_info(ctx.refine(ops, db, x, tol=1e-10, m=40, maxit=600))
    torch.cuda.synchronize()
    assert (st == 0).all() and (rr <= 1e-10).all(), (st, rr)
    for k in range(n):
        C = orc.coeffs(H, W, 0.02, 1e-3, 1 / H, mt[k])
        xr = x[k].cpu().numpy()
        assert np.linalg.norm(b[k] - orc.apply(H, W, C, xr)) <= 1.01e-10 * np.linalg.norm(b[k])


@pytest.mark.parametrize("minb", [4, 2])
def test_cluster_of_16_ctas_128x128(kp, orc, minb):
    # kp_options.cluster_size = 16: 128-thread CTAs of 8 columns (1024 points)
    # each, a non-portable cluster size, two or four systems' CTAs per SM;
    # the same tolerance and solutions as the 8-CTA default
    H = W = 128
    N = H * W
    rng = np.random.default_rng(16 + minb)
    n = 3
    mt = rng.uniform(0, 1, (n, N))
    b = rng.normal(size=(n, N))
    ctx = kp.Context(max_n=N, precision=kp.PREC_MIXED, cluster_size=16, cluster_blocks_per_sm=minb)
    dm, db = _dev(mt), _dev(b)
    ops = kp.make_ops(H, W, 1e-3, 0.02, 1 / H, dm)
    x = torch.zeros_like(db)
    it, st, rr = kp.decode_info(ctx.refine(ops, db, x, tol=1e-10, m=40, maxit=600))
    torch.cuda.synchronize()
    assert (st == 0).all() and (rr <= 1e-10).all(), (st, rr)
    for k in range(n):
        C = orc.coeffs(H, W, 0.02, 1e-3, 1 / H, mt[k])
        xr = x[k].cpu().numpy()
        assert np.linalg.norm(b[k] - orc.apply(H, W, C, xr)) <= 1.01e-10 * np.linalg.norm(b[k])
        ref = orc.gmres(H, W, C, b[k], tol=1e-13, m=40, maxit=800)
        assert np.linalg.norm(xr - ref.x) <= 1e-8 * np.linalg.norm(ref.x)
