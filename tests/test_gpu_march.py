"""The native time march (graph-replayed timesteps) against the oracle's
march, for the three initial-guess modes, one and several grid sizes."""
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


def _groups(wl):
    out = []
    for g in wl.groups:
        s = torch.as_tensor(g.seeds.reshape(len(g.seeds), -1).copy(), device="cuda")
        t = torch.as_tensor(g.targets.reshape(len(g.targets), -1).copy(), device="cuda")
        out.append((s, t, g.target_seed, g.H, g.W))
    return out


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
@pytest.mark.parametrize("use_graph", [True, False])
def test_march_matches_oracle_tiny(kp, orc, mode, use_graph):
    wl = synth.config(1)
    g = wl.groups[0]
    ctx = kp.Context(max_seeds=4, max_a=wl.a, max_n=g.N)
    grp = _groups(wl)
    mr = kp.March(ctx, grp, wl.T, wl.g2, mode=mode, tol_seed=1e-10, tol=1e-12, m_seed=wl.m_seed,
                  m=wl.m, maxit=1000, use_graph=use_graph)
    stats, _ = mr.run(0, 20, stats=True)
    stats2, _ = mr.run(20, wl.T - 20, stats=True)      # resume from the returned state
    torch.cuda.synchronize()
    oms, omt, ost = orc.march(g.H, g.W, wl.T, wl.g2, g.seeds, g.targets, g.target_seed,
                              mode=mode, tol_seed=1e-10, m_seed=wl.m_seed, a=wl.a, tol_ref=1e-12,
                              m_ref=wl.m)
    gt = grp[0][1].cpu().numpy()
    assert np.abs(gt - omt).max() <= 1e-9 * np.abs(omt).max()
    assert np.abs(grp[0][0].cpu().numpy() - oms).max() <= 1e-8 * np.abs(oms).max()
    allst = list(stats) + list(stats2)
    assert len(allst) == wl.T
    assert all(s.not_converged == 0 for s in allst)
    assert max(s.max_rel_res for s in allst) <= 1e-12
    gpu_it = np.array([s.tgt_iters for s in allst])
    orc_it = np.array([st.tgt_iters.sum() for st in ost])
    assert np.abs(gpu_it - orc_it).max() <= len(g.targets)       # at most +-1 per solve


def test_march_mixed_sizes_one_launch(kp, orc):
    # two grid sizes in one plan: all seeds in one launch, all targets in one
    gA = synth.make_group(77, 9, 11, 2, 2, 3, tag=1)
    gB = synth.make_group(78, 20, 16, 1, 1, 2, tag=2)
    T = 12
    g2 = synth.beta_schedule(T)
    wl = synth.Workload("mixed", T, g2, [gA, gB])
    ctx = kp.Context(max_seeds=16, max_a=30, max_n=400)
    grp = _groups(wl)
    mr = kp.March(ctx, grp, T, g2, mode=0, tol_seed=1e-10, tol=1e-12, m_seed=30, m=30)
    mr.run(0, T)
    torch.cuda.synchronize()
    for k, g in enumerate(wl.groups):
        oms, omt, _ = orc.march(g.H, g.W, T, g2, g.seeds, g.targets, g.target_seed,
                                tol_seed=1e-10, m_seed=30, a=30, tol_ref=1e-12, m_ref=30)
        assert np.abs(grp[k][1].cpu().numpy() - omt).max() <= 1e-9 * np.abs(omt).max()


def test_march_workload_32x32_sampled(kp, orc):
    # the benchmark's grid and launch configuration (32x32x3, 10 templates,
    # restart 40, tol 1e-8), over the first timesteps, all targets compared
    wl = synth.config(2, T=1000, ntargets=40)
    g = wl.groups[0]
    steps = 3
    ctx = kp.Context(max_seeds=2 * wl.n_seed_planes, max_a=wl.a, max_n=g.N)
    grp = _groups(wl)
    mr = kp.March(ctx, grp, wl.T, wl.g2, mode=0, tol_seed=wl.tol_seed, tol=wl.tol,
                  m_seed=wl.m_seed, m=wl.m)
    stats, tm = mr.run(0, steps, stats=True, timing=True)
    torch.cuda.synchronize()
    oms, omt, _ = orc.march(g.H, g.W, wl.T, wl.g2, g.seeds, g.targets, g.target_seed, steps=steps,
                            tol_seed=wl.tol_seed, m_seed=wl.m_seed, a=wl.a, tol_ref=wl.tol,
                            m_ref=wl.m)
    # both sides stop at 1e-8 relative residual; cond <= 1.1 here
    err = np.abs(grp[0][1].cpu().numpy() - omt).max() / np.abs(omt).max()
    assert err <= 1e-6
    assert all(s.max_rel_res <= 1e-8 for s in stats)
    assert tm.refine_ms > 0 and tm.launches == 3 * steps + 1


@pytest.mark.parametrize("mode,shape", [(0, (0, 0)), (1, (0, 0)), (0, (128, 3))])
def test_march_windows_bit_identical(kp, orc, mode, shape):
    # windows of K timesteps with dynamically claimed (timestep, system) items
    # compute every solve exactly as one launch per timestep does: the states,
    # iteration counts and residuals agree bit for bit, including ragged
    # windows and a run resumed in the middle of one
    wl = synth.config(2, T=1000, ntargets=48)
    g = wl.groups[0]
    steps = 21
    res = {}
    for K in (1, 8, 3):
        ctx = kp.Context(max_seeds=2 * K * wl.n_seed_planes, max_a=wl.a, max_n=g.N,
                         block_threads=shape[0], blocks_per_sm=shape[1])
        grp = _groups(wl)
        mr = kp.March(ctx, grp, wl.T, wl.g2, mode=mode, tol_seed=wl.tol_seed, tol=wl.tol,
                      m_seed=wl.m_seed, m=wl.m, window=K)
        st1, tm = mr.run(0, 5, stats=True, timing=True)
        st2, _ = mr.run(5, steps - 5, stats=True)
        torch.cuda.synchronize()
        nwin = -(-5 // K)
        assert tm.launches == 3 * nwin + 1
        res[K] = (grp[0][0].cpu().numpy(), grp[0][1].cpu().numpy(),
                  [(s.tgt_iters, s.seed_iters, s.max_rel_res) for s in list(st1) + list(st2)])
        mr.close()
        ctx.close()
    for K in (8, 3):
        assert np.array_equal(res[K][0], res[1][0])
        assert np.array_equal(res[K][1], res[1][1])
        assert res[K][2] == res[1][2]
    oms, omt, _ = orc.march(g.H, g.W, wl.T, wl.g2, g.seeds, g.targets, g.target_seed, steps=steps,
                            mode=mode, tol_seed=wl.tol_seed, m_seed=wl.m_seed, a=wl.a,
                            tol_ref=wl.tol, m_ref=wl.m)
    assert np.abs(res[8][1] - omt).max() / np.abs(omt).max() <= 1e-6


def test_march_windows_two_size_classes(kp, orc):
    # grids of <= 1024 points and larger ones in one plan: in window mode each
    # size class has its own solver shape and persistent launch (chained
    # programmatically); results match the oracle and do not depend on K
    gA = synth.make_group(91, 24, 24, 2, 2, 5, tag=1)
    gB = synth.make_group(92, 40, 40, 1, 1, 3, tag=2)
    T = 1000
    g2 = synth.beta_schedule(T)
    wl = synth.Workload("two-classes", T, g2, [gA, gB])
    steps = 20
    finals = {}
    for K in (8, 3):
        ctx = kp.Context(max_seeds=2 * K * 5, max_a=30, max_n=1600)
        grp = _groups(wl)
        mr = kp.March(ctx, grp, T, g2, mode=0, tol_seed=1e-10, tol=1e-12, m_seed=30, m=30, window=K)
        st, tm = mr.run(0, steps, stats=True, timing=True)
        assert tm.launches == 4 * (-(-steps // K)) + 1        # seeds + 2 classes + advance
        assert all(s.not_converged == 0 for s in st)
        finals[K] = [(x[0].cpu().numpy(), x[1].cpu().numpy()) for x in grp]
        mr.close()
        ctx.close()
    for a, b in zip(finals[8], finals[3]):
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    for k, g in enumerate(wl.groups):
        oms, omt, _ = orc.march(g.H, g.W, T, g2, g.seeds, g.targets, g.target_seed, steps=steps,
                                tol_seed=1e-10, m_seed=30, a=30, tol_ref=1e-12, m_ref=30)
        assert np.abs(finals[8][k][1] - omt).max() <= 1e-9 * np.abs(omt).max()


@pytest.mark.parametrize("window", [1, 4])
def test_march_score_and_embedding_match_oracle(kp, orc, window):
    # score of every solved timestep and the probability-flow embedding, fused
    # into the target solves, against the oracle's march_scores (whole
    # config-1 trajectory, per-timestep and windowed launches)
    wl = synth.config(1)
    g = wl.groups[0]
    steps = wl.T
    N = g.N
    nt = len(g.targets)
    ctx = kp.Context(max_seeds=2 * window * len(g.seeds) + 2, max_a=wl.a, max_n=N)
    grp = _groups(wl)
    score = torch.full((wl.T, nt, 2, N), float("nan"), dtype=torch.float64, device="cuda")
    emb = torch.zeros((nt, 2, N), dtype=torch.float64, device="cuda")
    mr = kp.March(ctx, grp, wl.T, wl.g2, mode=0, tol_seed=1e-10, tol=1e-12, m_seed=wl.m_seed,
                  m=wl.m, window=window, score=score, embed=emb)
    mr.run(0, 17)
    mr.run(17, steps - 17)
    torch.cuda.synchronize()
    _, omt, S, E = orc.march_scores(g.H, g.W, wl.T, wl.g2, g.seeds, g.targets, g.target_seed,
                                    steps=steps, tol_seed=1e-10, m_seed=wl.m_seed, a=wl.a,
                                    tol_ref=1e-12, m_ref=wl.m)
    sc = score.cpu().numpy()
    assert np.isfinite(sc).all()                      # every timestep written
    scale = np.abs(S).max()
    assert np.abs(sc - S).max() <= 1e-8 * scale
    assert np.abs(emb.cpu().numpy() - E).max() <= 1e-8 * np.abs(E).max()


def test_march_score_needs_both_buffers(kp):
    wl = synth.config(1)
    g = wl.groups[0]
    ctx = kp.Context(max_seeds=4, max_a=wl.a, max_n=g.N)
    score = torch.zeros((wl.T, len(g.targets), 2, g.N), dtype=torch.float64, device="cuda")
    with pytest.raises(kp.KPError):
        kp.March(ctx, _groups(wl), wl.T, wl.g2, score=score)


def test_march_exact_galerkin_sampled(kp, orc):
    # exact Galerkin initial guess (target's own operator) at the benchmark's
    # size and launch configuration (windows, 128x4 shape), against the oracle
    wl = synth.config(2, T=1000, ntargets=24)
    g = wl.groups[0]
    steps = 5
    ctx = kp.Context(max_seeds=2 * 8 * wl.n_seed_planes, max_a=wl.a, max_n=g.N)
    grp = _groups(wl)
    mr = kp.March(ctx, grp, wl.T, wl.g2, mode=3, tol_seed=wl.tol_seed, tol=1e-10,
                  m_seed=wl.m_seed, m=wl.m, window=8)
    st, _ = mr.run(0, steps, stats=True)
    torch.cuda.synchronize()
    _, omt, ost = orc.march(g.H, g.W, wl.T, wl.g2, g.seeds, g.targets, g.target_seed, steps=steps,
                            mode=3, tol_seed=wl.tol_seed, m_seed=wl.m_seed, a=wl.a, tol_ref=1e-10,
                            m_ref=wl.m)
    assert np.abs(grp[0][1].cpu().numpy() - omt).max() <= 1e-8 * np.abs(omt).max()
    gpu_it = np.array([s.tgt_iters for s in st])
    orc_it = np.array([o.tgt_iters.sum() for o in ost])
    assert np.abs(gpu_it - orc_it).max() <= len(g.targets)


@pytest.mark.parametrize("window", [1, 4])
def test_march_picard_iterations_match_oracle(kp, orc, window):
    # K = 3 Picard iterations per timestep (lagged term on the latest iterate)
    # for seeds and targets, whole config-1 trajectory, against the oracle
    wl = synth.config(1)
    g = wl.groups[0]
    ctx = kp.Context(max_seeds=2 * window * len(g.seeds) + 2, max_a=wl.a, max_n=g.N)
    grp = _groups(wl)
    mr = kp.March(ctx, grp, wl.T, wl.g2, mode=0, tol_seed=1e-11, tol=1e-12, m_seed=wl.m_seed,
                  m=wl.m, window=window, picard=3)
    st, _ = mr.run(0, wl.T, stats=True)
    torch.cuda.synchronize()
    oms, omt, _ = orc.march(g.H, g.W, wl.T, wl.g2, g.seeds, g.targets, g.target_seed,
                            tol_seed=1e-11, m_seed=wl.m_seed, a=wl.a, tol_ref=1e-12, m_ref=wl.m,
                            picard=3)
    assert np.abs(grp[0][1].cpu().numpy() - omt).max() <= 1e-9 * np.abs(omt).max()
    assert np.abs(grp[0][0].cpu().numpy() - oms).max() <= 1e-9 * np.abs(oms).max()
    # the extra iterations ran (more steps than one solve per timestep) and
    # moved the answer (the lagged term changed)
    _, mt1, one = orc.march(g.H, g.W, wl.T, wl.g2, g.seeds, g.targets, g.target_seed,
                            tol_seed=1e-11, m_seed=wl.m_seed, a=wl.a, tol_ref=1e-12, m_ref=wl.m)
    assert sum(s.tgt_iters for s in st) > sum(o.tgt_iters.sum() for o in one)
    assert np.abs(omt - mt1).max() > 1e-12 * np.abs(omt).max()


def test_march_without_seeds_windowed(kp, orc):
    # a plan of targets only (plain GMRES from zero, no seed chains, windows
    # of 4 timesteps and a ragged last window) against the oracle
    g = synth.make_group(95, 20, 18, 2, 1, 6, tag=3)
    T = 30
    g2 = synth.beta_schedule(T)
    ctx = kp.Context(max_seeds=1, max_a=30, max_n=g.N)
    s = torch.zeros((0, g.N), dtype=torch.float64, device="cuda")
    t = torch.as_tensor(g.targets.reshape(len(g.targets), -1).copy(), device="cuda")
    mr = kp.March(ctx, [(s, t, np.zeros(len(t), np.int32), g.H, g.W)], T, g2, mode=1,
                  tol=1e-12, m=30, window=4)
    st, tm = mr.run(0, T, stats=True, timing=True)
    torch.cuda.synchronize()
    assert tm.launches == 2 * (-(-T // 4))                 # target launch + advance per window
    _, omt, _ = orc.march(g.H, g.W, T, g2, g.seeds[:1], g.targets, np.zeros(len(t), np.int32),
                          mode=1, tol_ref=1e-12, m_ref=30)
    assert np.abs(t.cpu().numpy() - omt).max() <= 1e-9 * np.abs(omt).max()
    assert all(x.seed_iters == 0 for x in st)


@pytest.mark.parametrize("window", [1, 0])
def test_march_bicgstab_seeds_match_oracle(kp, orc, window):
    # the paper's Phase 1: BiCGSTAB seeds, their key vectors as the basis and
    # the explicit A_proj for the targets, against the oracle's march
    wl = synth.config(1)
    g = wl.groups[0]
    ctx = kp.Context(max_seeds=8, max_a=wl.a, max_n=g.N)
    grp = _groups(wl)
    mr = kp.March(ctx, grp, wl.T, wl.g2, mode=0, tol_seed=1e-12, tol=1e-12, m_seed=wl.m_seed,
                  m=wl.m, maxit=1000, window=window, seed_solver=kp.SEED_BICGSTAB)
    stats, _ = mr.run(0, wl.T, stats=True)
    torch.cuda.synchronize()
    oms, omt, ost = orc.march(g.H, g.W, wl.T, wl.g2, g.seeds, g.targets, g.target_seed,
                              mode=0, tol_seed=1e-12, m_seed=wl.m_seed, a=wl.a, tol_ref=1e-12,
                              m_ref=wl.m, seed_solver=orc.SEED_BICGSTAB)
    assert np.abs(grp[0][1].cpu().numpy() - omt).max() <= 1e-9 * np.abs(omt).max()
    assert np.abs(grp[0][0].cpu().numpy() - oms).max() <= 1e-9 * np.abs(oms).max()
    assert all(s.not_converged == 0 for s in stats)
    assert max(s.max_rel_res for s in stats) <= 1e-12
    # the projected guesses are the oracle's: the refine needs as many steps
    gpu_it = np.array([s.tgt_iters for s in stats])
    orc_it = np.array([st.tgt_iters.sum() for st in ost])
    assert np.abs(gpu_it - orc_it).max() <= len(g.targets)
    seed_it = np.array([s.seed_iters for s in stats])
    orc_sit = np.array([st.seed_iters.sum() for st in ost])
    assert np.abs(seed_it - orc_sit).max() <= len(g.seeds)


def test_march_bicgstab_seeds_32x32_windowed(kp, orc):
    # the benchmark's grid and launch shape with BiCGSTAB seeds, windows of 4
    wl = synth.config(2, T=1000, ntargets=40)
    g = wl.groups[0]
    steps = 8
    ctx = kp.Context(max_seeds=8 * wl.n_seed_planes, max_a=wl.a, max_n=g.N)
    grp = _groups(wl)
    mr = kp.March(ctx, grp, wl.T, wl.g2, mode=0, tol_seed=wl.tol_seed, tol=wl.tol,
                  m_seed=wl.m_seed, m=wl.m, window=4, seed_solver=kp.SEED_BICGSTAB)
    stats, _ = mr.run(0, steps, stats=True)
    torch.cuda.synchronize()
    assert all(s.max_rel_res <= 1e-8 and s.not_converged == 0 for s in stats)
    oms, omt, ost = orc.march(g.H, g.W, wl.T, wl.g2, g.seeds, g.targets, g.target_seed, steps=steps,
                              tol_seed=wl.tol_seed, m_seed=wl.m_seed, a=wl.a, tol_ref=wl.tol,
                              m_ref=wl.m, seed_solver=orc.SEED_BICGSTAB)
    assert np.abs(grp[0][1].cpu().numpy() - omt).max() <= 1e-6 * np.abs(omt).max()
    gpu_it = np.array([s.tgt_iters for s in stats])
    orc_it = np.array([st.tgt_iters.sum() for st in ost])
    assert np.abs(gpu_it - orc_it).max() <= len(g.targets)


def test_march_bicgstab_seeds_rejected_combinations(kp):
    wl = synth.config(1)
    g = wl.groups[0]
    grp = _groups(wl)
    ctx = kp.Context(max_seeds=8, max_a=wl.a, max_n=g.N)
    with pytest.raises(RuntimeError):
        kp.March(ctx, grp, wl.T, wl.g2, mode=0, picard=2, seed_solver=kp.SEED_BICGSTAB)
    with pytest.raises(RuntimeError):
        kp.March(ctx, grp, wl.T, wl.g2, mode=0, seed_solver=7)
    mctx = kp.Context(max_seeds=8, max_a=wl.a, max_n=g.N, precision=kp.PREC_MIXED)
    with pytest.raises(RuntimeError):
        kp.March(mctx, grp, wl.T, wl.g2, mode=0, seed_solver=kp.SEED_BICGSTAB)


def _chains(ntemplates, channels):
    # seed k*channels + ch extends seed (k-1)*channels + ch: one chain per channel
    return np.array([(k - 1) * channels + ch if k > 0 else -1
                     for k in range(ntemplates) for ch in range(channels)], dtype=np.int32)


@pytest.mark.parametrize("window,solver", [(1, 0), (0, 0), (0, 1)])
def test_march_seed_cycling_matches_oracle(kp, orc, window, solver):
    # seed cycling (Sec. 5.2): every seed with a predecessor serves its own
    # basis followed by the predecessor's served one, with its own A_proj
    g = synth.make_group(91, 12, 10, 2, 3, 6, tag=3)
    T = 12
    g2 = synth.beta_schedule(T)
    prev = _chains(3, 2)
    ctx = kp.Context(max_seeds=48, max_a=20, max_n=g.N)
    s = torch.as_tensor(g.seeds.reshape(len(g.seeds), -1).copy(), device="cuda")
    t = torch.as_tensor(g.targets.reshape(len(g.targets), -1).copy(), device="cuda")
    mr = kp.March(ctx, [(s, t, g.target_seed, g.H, g.W, prev)], T, g2, mode=0, tol_seed=1e-12,
                  tol=1e-12, m_seed=20, m=20, maxit=1000, window=window, seed_solver=solver)
    stats, _ = mr.run(0, T, stats=True)
    torch.cuda.synchronize()
    oms, omt, ost = orc.march(g.H, g.W, T, g2, g.seeds, g.targets, g.target_seed, mode=0,
                              tol_seed=1e-12, m_seed=20, a=20, tol_ref=1e-12, m_ref=20,
                              seed_solver=solver, seed_prev=prev)
    assert np.abs(t.cpu().numpy() - omt).max() <= 1e-9 * np.abs(omt).max()
    assert np.abs(s.cpu().numpy() - oms).max() <= 1e-9 * np.abs(oms).max()
    assert all(x.not_converged == 0 and x.max_rel_res <= 1e-12 for x in stats)
    gpu_it = np.array([x.tgt_iters for x in stats])
    orc_it = np.array([x.tgt_iters.sum() for x in ost])
    assert np.abs(gpu_it - orc_it).max() <= len(g.targets)


def test_march_seed_cycling_32x32_windowed(kp, orc):
    # the benchmark's workload with one chain of the ten template seeds per
    # channel, windows of 4, against the oracle's cycling march
    wl = synth.config(2, T=1000, ntargets=40)
    g = wl.groups[0]
    steps = 8
    prev = _chains(10, 3)
    ctx = kp.Context(max_seeds=8 * wl.n_seed_planes, max_a=wl.a, max_n=g.N)
    s = torch.as_tensor(g.seeds.reshape(len(g.seeds), -1).copy(), device="cuda")
    t = torch.as_tensor(g.targets.reshape(len(g.targets), -1).copy(), device="cuda")
    mr = kp.March(ctx, [(s, t, g.target_seed, g.H, g.W, prev)], wl.T, wl.g2, mode=0,
                  tol_seed=wl.tol_seed, tol=wl.tol, m_seed=wl.m_seed, m=wl.m, window=4)
    stats, _ = mr.run(0, steps, stats=True)
    torch.cuda.synchronize()
    assert all(x.max_rel_res <= 1e-8 and x.not_converged == 0 for x in stats)
    oms, omt, ost = orc.march(g.H, g.W, wl.T, wl.g2, g.seeds, g.targets, g.target_seed, steps=steps,
                              tol_seed=wl.tol_seed, m_seed=wl.m_seed, a=wl.a, tol_ref=wl.tol,
                              m_ref=wl.m, seed_prev=prev)
    assert np.abs(t.cpu().numpy() - omt).max() <= 1e-6 * np.abs(omt).max()
    gpu_it = np.array([x.tgt_iters for x in stats])
    orc_it = np.array([x.tgt_iters.sum() for x in ost])
    assert np.abs(gpu_it - orc_it).max() <= len(g.targets)


def test_march_seed_cycling_rejects_bad_links(kp):
    g = synth.make_group(91, 12, 10, 2, 3, 6, tag=3)
    ctx = kp.Context(max_seeds=48, max_a=20, max_n=g.N)
    s = torch.as_tensor(g.seeds.reshape(len(g.seeds), -1).copy(), device="cuda")
    t = torch.as_tensor(g.targets.reshape(len(g.targets), -1).copy(), device="cuda")
    bad = np.array([-1, 0, 2, 1, 2, 3], dtype=np.int32)           # seed 2 names itself
    with pytest.raises(RuntimeError):
        kp.March(ctx, [(s, t, g.target_seed, g.H, g.W, bad)], 12, synth.beta_schedule(12))


def test_march_bounded_wait_gives_up_and_context_survives(kp, orc):
    # every target item waits for a release that never comes (testing aid):
    # the waits give up, the run reports KP_ERR_TIMEOUT, and a normal plan on
    # the same context afterwards still matches the oracle
    wl = synth.config(1)
    g = wl.groups[0]
    ctx = kp.Context(max_seeds=8, max_a=wl.a, max_n=g.N)
    grp = _groups(wl)
    bad = kp.March(ctx, grp, wl.T, wl.g2, mode=0, tol_seed=1e-10, tol=1e-12, m_seed=wl.m_seed,
                   m=wl.m, window=2, wait_probe=True)
    with pytest.raises(kp.KPError) as ei:
        bad.run(0, 4, stats=True)
    assert ei.value.status == kp.ERR_TIMEOUT
    bad.close()
    grp = _groups(wl)
    mr = kp.March(ctx, grp, wl.T, wl.g2, mode=0, tol_seed=1e-10, tol=1e-12, m_seed=wl.m_seed,
                  m=wl.m, window=2)
    stats, _ = mr.run(0, 6, stats=True)
    torch.cuda.synchronize()
    oms, omt, _ = orc.march(g.H, g.W, wl.T, wl.g2, g.seeds, g.targets, g.target_seed, steps=6,
                            mode=0, tol_seed=1e-10, m_seed=wl.m_seed, a=wl.a, tol_ref=1e-12,
                            m_ref=wl.m)
    assert np.abs(grp[0][1].cpu().numpy() - omt).max() <= 1e-9 * np.abs(omt).max()
    assert all(s.not_converged == 0 for s in stats)


def test_march_seed_cycling_4096_point_grid(kp, orc):
    # the cycling kernel's 16-points-per-thread instance (grids of 1025..4096
    # points) on a 64x64 chain of three seeds, against the oracle
    g = synth.make_group(93, 64, 64, 1, 3, 4, tag=5)
    T = 6
    g2 = synth.beta_schedule(T)
    prev = _chains(3, 1)
    ctx = kp.Context(max_seeds=12, max_a=20, max_n=g.N)
    s = torch.as_tensor(g.seeds.reshape(len(g.seeds), -1).copy(), device="cuda")
    t = torch.as_tensor(g.targets.reshape(len(g.targets), -1).copy(), device="cuda")
    mr = kp.March(ctx, [(s, t, g.target_seed, g.H, g.W, prev)], T, g2, mode=0, tol_seed=1e-12,
                  tol=1e-12, m_seed=20, m=20, maxit=1000, window=2)
    stats, _ = mr.run(0, T, stats=True)
    torch.cuda.synchronize()
    oms, omt, ost = orc.march(g.H, g.W, T, g2, g.seeds, g.targets, g.target_seed, mode=0,
                              tol_seed=1e-12, m_seed=20, a=20, tol_ref=1e-12, m_ref=20,
                              seed_prev=prev)
    assert np.abs(t.cpu().numpy() - omt).max() <= 1e-9 * np.abs(omt).max()
    assert all(x.not_converged == 0 and x.max_rel_res <= 1e-12 for x in stats)
    gpu_it = np.array([x.tgt_iters for x in stats])
    orc_it = np.array([x.tgt_iters.sum() for x in ost])
    assert np.abs(gpu_it - orc_it).max() <= len(g.targets)


def test_march_combined_options_match_oracle(kp, orc):
    # options that share the feature variant of the solver: seed cycling with
    # the score / embedding output, and the exact Galerkin guess on BiCGSTAB
    # seed bases, each against the oracle's march
    g = synth.make_group(91, 12, 10, 2, 3, 6, tag=3)
    T = 10
    g2 = synth.beta_schedule(T)
    prev = _chains(3, 2)
    N, nt = g.N, len(g.targets)
    ctx = kp.Context(max_seeds=48, max_a=20, max_n=N)
    s = torch.as_tensor(g.seeds.reshape(len(g.seeds), -1).copy(), device="cuda")
    t = torch.as_tensor(g.targets.reshape(len(g.targets), -1).copy(), device="cuda")
    score = torch.full((T, nt, 2, N), float("nan"), dtype=torch.float64, device="cuda")
    emb = torch.zeros((nt, 2, N), dtype=torch.float64, device="cuda")
    mr = kp.March(ctx, [(s, t, g.target_seed, g.H, g.W, prev)], T, g2, mode=0, tol_seed=1e-12,
                  tol=1e-12, m_seed=20, m=20, window=2, score=score, embed=emb)
    mr.run(0, T)
    torch.cuda.synchronize()
    _, omt, S, E = orc.march_scores(g.H, g.W, T, g2, g.seeds, g.targets, g.target_seed, mode=0,
                                    tol_seed=1e-12, m_seed=20, a=20, tol_ref=1e-12, m_ref=20,
                                    seed_prev=prev)
    assert np.abs(t.cpu().numpy() - omt).max() <= 1e-9 * np.abs(omt).max()
    assert np.abs(score.cpu().numpy() - S).max() <= 1e-8 * np.abs(S).max()
    assert np.abs(emb.cpu().numpy() - E).max() <= 1e-8 * np.abs(E).max()

    s = torch.as_tensor(g.seeds.reshape(len(g.seeds), -1).copy(), device="cuda")
    t = torch.as_tensor(g.targets.reshape(len(g.targets), -1).copy(), device="cuda")
    mr = kp.March(ctx, [(s, t, g.target_seed, g.H, g.W)], T, g2, mode=kp.MARCH_GALERKIN,
                  tol_seed=1e-12, tol=1e-12, m_seed=20, m=20, window=2,
                  seed_solver=kp.SEED_BICGSTAB)
    stats, _ = mr.run(0, T, stats=True)
    torch.cuda.synchronize()
    _, omt, ost = orc.march(g.H, g.W, T, g2, g.seeds, g.targets, g.target_seed, mode=3,
                            tol_seed=1e-12, m_seed=20, a=20, tol_ref=1e-12, m_ref=20,
                            seed_solver=orc.SEED_BICGSTAB)
    assert np.abs(t.cpu().numpy() - omt).max() <= 1e-9 * np.abs(omt).max()
    gpu_it = np.array([x.tgt_iters for x in stats])
    orc_it = np.array([x.tgt_iters.sum() for x in ost])
    assert np.abs(gpu_it - orc_it).max() <= nt
