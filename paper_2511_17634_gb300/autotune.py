"""Autotuner for the time march: picks the GMRES restart length m and the
shared-memory Krylov window (which sets how many blocks share an SM) for a
workload by timing a few calibration timesteps of the real march, and caches
the choice in a JSON file keyed by (device, grid sizes, batch, precision).

Candidates: m in {20, 30, 40, 60} x shared-memory window in {auto, small} x
(threads per system, resident blocks per SM) in {(256, 2), (128, 3), (128, 4),
(64, 4)} (FP64 grids of up to 1024 points; one shape otherwise).
The timing runs through the C ABI (kp_march_*) on the GPU; only the choice of
the fastest candidate and the cache are host logic.
"""
from __future__ import annotations

import json
import os

M_CANDIDATES = (20, 30, 40, 60)
WINDOW_CANDIDATES = (0, 6)      # 0 = automatic (two blocks per SM when N <= 1024)
SHAPE_CANDIDATES = ((256, 2), (128, 3), (128, 4), (64, 4))   # (threads, blocks per SM), N <= 1024


def cache_key(device: str, grids, nseed: int, ntgt: int, precision: str, mode: int) -> str:
    g = ",".join(f"{h}x{w}" for h, w in grids)
    return f"{device}|{g}|s{nseed}|t{ntgt}|{precision}|mode{mode}"


def load_cache(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(path: str, cache: dict) -> None:
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def choose(timings: dict):
    """Fastest candidate of {(m, window, threads): seconds}; ties go to the smaller m."""
    return min(timings.items(), key=lambda kv: (kv[1],) + tuple(kv[0]))[0]


def tune(wl, mode=0, steps=4, cache_path=None, time_fn=None):
    """Returns {'m', 'smem_vectors', 'block_threads', 'blocks_per_sm', 'timings'}
    for workload `wl` (synth.Workload).  time_fn(m, S, (threads, blocks per SM))
    -> seconds overrides the GPU timing."""
    precision = wl.precision
    if time_fn is None:
        import torch
        device = torch.cuda.get_device_name()
    else:
        device = "fake"
    key = cache_key(device, [(g.H, g.W) for g in wl.groups], wl.n_seed_planes,
                    wl.n_target_planes, precision, mode)
    cache = load_cache(cache_path) if cache_path else {}
    if key in cache:
        return cache[key]
    if time_fn is None:
        time_fn = _gpu_timer(wl, mode, steps)
    small = max(g.N for g in wl.groups) <= 1024 and precision != "mixed"
    shapes = SHAPE_CANDIDATES if small else ((0, 0),)
    timings = {}
    for m in M_CANDIDATES:
        for S in WINDOW_CANDIDATES:
            for sh in shapes:
                timings[(m, S, sh)] = time_fn(m, S, sh)
    m, S, (nt, mb) = choose(timings)
    res = {"m": m, "smem_vectors": S, "block_threads": nt, "blocks_per_sm": mb,
           "timings": {f"m{a}_S{b}_t{c[0]}x{c[1]}": t for (a, b, c), t in timings.items()}}
    if cache_path:
        cache[key] = res
        save_cache(cache_path, cache)
    return res


def _gpu_timer(wl, mode, steps):
    import torch

    from . import kp

    dev = torch.device("cuda", torch.cuda.current_device())
    seeds = [torch.as_tensor(g.seeds.reshape(len(g.seeds), -1), device=dev) for g in wl.groups]
    tgts = [torch.as_tensor(g.targets.reshape(len(g.targets), -1), device=dev) for g in wl.groups]
    nmax = max(g.N for g in wl.groups)
    prec = kp.PREC_MIXED if wl.precision == "mixed" else kp.PREC_FP64

    # the march the workload will run: windows of 16 timesteps in FP64 (one
    # per launch in mixed precision), the workload's basis length a
    window = 1 if wl.precision == "mixed" else 16

    def run(m, S, shape):
        ctx = kp.Context(max_seeds=max(2 * window * wl.n_seed_planes, 1), max_a=wl.a, max_n=nmax,
                         precision=prec, smem_vectors=S, block_threads=shape[0],
                         blocks_per_sm=shape[1])
        ss = [x.clone() for x in seeds]
        tt = [x.clone() for x in tgts]
        groups = [(ss[k], tt[k], g.target_seed, g.H, g.W) for k, g in enumerate(wl.groups)]
        plan = kp.March(ctx, groups, wl.T, wl.g2, mode=mode, tol_seed=wl.tol_seed, tol=wl.tol,
                        m_seed=wl.m_seed, m=m, maxit=1000, window=window)
        plan.run(0, steps)                       # warm-up (graphs, caches)
        best = float("inf")
        for _ in range(2):
            for a, b in zip(ss, seeds):
                a.copy_(b)
            for a, b in zip(tt, tgts):
                a.copy_(b)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            plan.run(0, steps)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1000.0)
        plan.close()
        ctx.close()
        return best

    return run
