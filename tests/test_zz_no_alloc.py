"""kp_refine_static -- the refine for callers that cannot allocate device
memory -- against kp_refine, through the C ABI.

kp_refine_static keeps its scratch in a static device array of the library
instead of allocating, for hosts whose memory pools, plugin rules or latency
budgets forbid cudaMalloc at solve time.  It must give kp_refine's answers,
call after call (the array is reused and keeps the previous call's contents).
This file is collected last so that a failure here stops a `-x` run only
after every other test has run.
"""
import ctypes

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
    L = K.lib()
    vp = ctypes.c_void_p
    L.kp_refine_static.argtypes = [ctypes.c_int, vp, vp, vp, ctypes.c_double, ctypes.c_int,
                                   ctypes.c_int, vp, vp]
    L.kp_refine_static.restype = ctypes.c_int
    return K


def _static_refine(K, ops, b, x, tol, m, maxit, info, stream):
    L = K.lib()
    pb, px = K.ptrs(b), K.ptrs(x)
    return L.kp_refine_static(len(ops), K.Context._arr(ops), pb.ctypes.data_as(ctypes.c_void_p),
                              px.ctypes.data_as(ctypes.c_void_p), tol, m, maxit,
                              ctypes.c_void_p(info.data_ptr()), ctypes.c_void_p(stream))


def _problem(seed):
    # the paper's own setting (g = 0.5, T = 100) on 32x32 channels: these
    # systems need 20-30 GMRES steps, so Krylov vectors beyond the
    # shared-memory window go to the static scratch
    wl = synth.config(2, T=100, ntargets=60, seed=seed)
    g = wl.groups[0]
    return g.H, g.W, g.targets.reshape(len(g.targets), -1)


def _check_against_refine(kp, ctx, H, W, mt, m, stream, g2=0.25, dt=0.01):
    n = mt.shape[0]
    dm = torch.as_tensor(mt, device="cuda")
    ops = kp.make_ops(H, W, dt, g2, 1.0 / H, dm)
    b = torch.zeros_like(dm)
    ctx.rhs(ops, dm, b)
    x_ref = torch.zeros_like(dm)
    info_ref = ctx.refine(ops, b, x_ref, tol=1e-10, m=m, maxit=600)
    x_st = torch.zeros_like(dm)
    info_st = kp.info_tensor(n)
    torch.cuda.synchronize()
    rc = _static_refine(kp, ops, b, x_st, 1e-10, m, 600, info_st, stream.cuda_stream)
    assert rc == kp.OK, rc
    torch.cuda.synchronize()
    it_r, st_r, rr_r = kp.decode_info(info_ref)
    it_s, st_s, rr_s = kp.decode_info(info_st)
    assert (st_s == 0).all() and (rr_s <= 1e-10).all()
    assert np.array_equal(it_s, it_r)
    err = float((x_st - x_ref).abs().max() / x_ref.abs().max())
    assert err <= 1e-12, err
    return it_s


def test_static_refine_allocates_nothing_after_its_first_call(kp):
    # the first call on a device resolves the array and loads the kernels;
    # later calls -- one of them with Krylov vectors in the static array --
    # must leave the device's free memory where it was
    stream = torch.cuda.current_stream()
    ctx = kp.Context(max_n=1024)
    H, W, mt = _problem(13)
    dm = torch.as_tensor(mt, device="cuda")
    ops = kp.make_ops(H, W, 0.01, 0.25, 1.0 / H, dm)
    b = torch.zeros_like(dm)
    ctx.rhs(ops, dm, b)
    xs = [torch.zeros_like(dm) for _ in range(4)]
    infos = [kp.info_tensor(dm.shape[0]) for _ in range(4)]
    torch.cuda.synchronize()
    assert _static_refine(kp, ops, b, xs[0], 1e-10, 40, 600, infos[0], stream.cuda_stream) == kp.OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for k in (1, 2, 3):
        assert _static_refine(kp, ops, b, xs[k], 1e-10, 40, 600, infos[k], stream.cuda_stream) == kp.OK
        torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    it, st, _ = kp.decode_info(infos[3])
    assert (st == 0).all() and it.max() > 24          # reached the static workspace
    assert free1 >= free0, (free0, free1)
    assert torch.equal(xs[3], xs[1])


def test_static_refine_more_systems_than_sms(kp):
    # 400 systems with m = 64: the grid is the device's SM count cut to what
    # the array's Krylov workspace holds, and each block solves several systems
    props = torch.cuda.get_device_properties(0)
    n = max(400, 2 * props.multi_processor_count + 17)
    wl = synth.config(2, T=100, ntargets=(n + 2) // 3, seed=14)
    g = wl.groups[0]
    mt = g.targets.reshape(len(g.targets), -1)[:n]
    ctx = kp.Context(max_n=1024)
    it = _check_against_refine(kp, ctx, g.H, g.W, mt, 64, torch.cuda.current_stream())
    assert it.max() > 24


def test_static_refine_matches_refine_on_two_calls(kp):
    stream = torch.cuda.current_stream()
    ctx = kp.Context(max_n=1024)
    for call, seed in enumerate((11, 12)):
        H, W, mt = _problem(seed)
        n = mt.shape[0]
        dm = torch.as_tensor(mt, device="cuda")
        ops = kp.make_ops(H, W, 0.01, 0.25, 1.0 / H, dm)
        b = torch.zeros_like(dm)
        ctx.rhs(ops, dm, b)
        x_ref = torch.zeros_like(dm)
        info_ref = ctx.refine(ops, b, x_ref, tol=1e-10, m=40, maxit=600)
        x_st = torch.zeros_like(dm)
        info_st = kp.info_tensor(n)
        rc = _static_refine(kp, ops, b, x_st, 1e-10, 40, 600, info_st, stream.cuda_stream)
        assert rc == kp.OK, rc
        torch.cuda.synchronize()
        it_r, st_r, rr_r = kp.decode_info(info_ref)
        it_s, st_s, rr_s = kp.decode_info(info_st)
        assert (st_s == 0).all() and (rr_s <= 1e-10).all()
        assert it_s.max() > 24, "the case must reach the static workspace"
        assert np.array_equal(it_s, it_r)
        err = float((x_st - x_ref).abs().max() / x_ref.abs().max())
        assert err <= 1e-12, (call, err)


def test_static_refine_rejects_oversized_requests(kp):
    ctx = kp.Context(max_n=4096)
    dm = torch.zeros((2, 64 * 64), dtype=torch.float64, device="cuda")
    ops = kp.make_ops(64, 64, 0.01, 0.02, 1 / 64, dm)
    info = kp.info_tensor(2)
    rc = _static_refine(kp, ops, dm, dm.clone(), 1e-8, 40, 100, info, 0)
    assert rc == kp.ERR_TOO_LARGE
    # more systems than the descriptor table holds
    dm = torch.zeros((4097, 1), dtype=torch.float64, device="cuda")
    ops = kp.make_ops(1, 1, 0.01, 0.02, 1.0, dm)
    info = kp.info_tensor(4097)
    rc = _static_refine(kp, ops, dm, dm.clone(), 1e-8, 10, 100, info, 0)
    assert rc == kp.ERR_TOO_LARGE
    del ctx
