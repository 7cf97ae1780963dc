"""Learned initial guess for the target solves (not in the paper).

A small 3x3 convolutional network (kp.CNN, trained with the library's own
tensor-core kernels) predicts the correction Delta = m_i^n - m_seed^n from
[target image, seed state m_seed^n, time embedding]; the target's initial
guess is X_init = m_seed^n + Delta, projected in residual form onto the seed's
Krylov basis (x0 = X_init + V_a H_a^{-1} V_a^T (b - A X_init), Sec. 3 Phase 2)
and refined by GMRES to the same tolerance as every other solve, so the
network can only change the cost of a solve, never its accuracy.

Host orchestration only: every arithmetic step runs in the CUDA library.
"""
from __future__ import annotations

import numpy as np

from . import kp

CHANNELS = (6, 32, 32, 32, 1)


def init_params(seed=0, channels=CHANNELS):
    """He-style initial weights, small biases, in the network's flat layout."""
    rng = np.random.default_rng(seed)
    parts = []
    for ci, co in zip(channels[:-1], channels[1:]):
        parts.append(rng.normal(scale=np.sqrt(2.0 / (9 * ci)), size=co * ci * 9))
        parts.append(np.zeros(co))
    p = np.concatenate(parts)
    # start the last layer near zero so that X_init starts at m_seed^n
    nlast = channels[-2] * 9 * channels[-1]
    p[-(nlast + channels[-1]):-channels[-1]] *= 0.01
    return p.astype(np.float32)


def generate_pairs(ctx, net, group, T, g2, steps, every, tol_seed=1e-10, tol=1e-8, m=40):
    """Run the method (projected march) over `steps` timesteps for the group's
    seeds and targets and, every `every` steps, record the network input and
    target m_i^n - m_seed^n of every target channel.  Returns float32 CUDA
    tensors (inputs [n][6][P], targets [n][1][P])."""
    import torch
    H, W = group.H, group.W
    P = H * W
    dev = torch.device("cuda", torch.cuda.current_device())
    img = torch.as_tensor(group.targets.reshape(len(group.targets), -1).copy(), device=dev)
    s = torch.as_tensor(group.seeds.reshape(len(group.seeds), -1).copy(), device=dev)
    t = img.clone()
    plan = kp.March(ctx, [(s, t, group.target_seed, H, W)], T, g2, mode=kp.MARCH_PROJECTED,
                    tol_seed=tol_seed, tol=tol, m_seed=m, m=m)
    ins, outs = [], []
    n = 0
    nt = t.shape[0]
    seed_rows = [s[int(k)] for k in group.target_seed]
    while n + every <= steps:
        plan.run(n, every)
        n += every
        x = torch.empty((nt, 6, P), dtype=torch.float32, device=dev)
        y = torch.empty((nt, 1, P), dtype=torch.float32, device=dev)
        net.pack_inputs([img[k] for k in range(nt)], seed_rows, n / T, x)
        net.pack_target([t[k] for k in range(nt)], seed_rows, y)
        ins.append(x)
        outs.append(y)
    plan.close()
    return torch.cat(ins), torch.cat(outs)


def train(net, inputs, targets, epochs, batch, lr=1e-3, seed=0):
    """Adam over shuffled mini-batches; returns the mean loss of every epoch."""
    import torch
    g = torch.Generator(device="cpu").manual_seed(seed)
    n = inputs.shape[0]
    t = 0
    hist = []
    for _ in range(epochs):
        perm = torch.randperm(n, generator=g)
        tot = 0.0
        nb = 0
        for k in range(0, n - batch + 1, batch):
            idx = perm[k:k + batch].to(inputs.device)
            t += 1
            tot += net.train_step(inputs.index_select(0, idx).contiguous(),
                                  targets.index_select(0, idx).contiguous(), t, lr=lr)
            nb += 1
        hist.append(tot / max(nb, 1))
    return hist


def step_compare(ctx, net, group, T, g2, n, seeds_prev, tgt_prev, tol_seed=1e-10, tol=1e-8, m=40,
                 slot_base=0):
    """Timestep n (1-based) for targets whose m^{n-1} is tgt_prev and seeds
    whose m^{n-1} is seeds_prev (CUDA [k][P] FP64).  Solves it three ways and
    returns ({mode: (initial relative residuals, Arnoldi steps, solutions),
    'times': {mode: seconds of the target-side work}}, seed solutions) for
    'projected' (paper), 'learned' and 'plain' (x0 = 0)."""
    import torch
    H, W = group.H, group.W
    dt, h, gg = 1.0 / T, 1.0 / H, float(g2[n - 1])
    img = torch.as_tensor(group.targets.reshape(len(group.targets), -1).copy(),
                          device=tgt_prev.device)
    nt = tgt_prev.shape[0]
    sops = kp.make_ops(H, W, dt, gg, h, seeds_prev)
    sb = torch.empty_like(seeds_prev)
    ctx.rhs(sops, seeds_prev, sb)
    sx = torch.zeros_like(seeds_prev)
    ctx.seed_solve(sops, sb, sx, tol=tol_seed, m=m, maxit=1000)
    for k in range(seeds_prev.shape[0]):
        ctx.store_basis(slot_base + k, n, k)
    tops = kp.make_ops(H, W, dt, gg, h, tgt_prev)
    tb = torch.empty_like(tgt_prev)
    ctx.rhs(tops, tgt_prev, tb)
    slots = np.asarray(group.target_seed, dtype=np.int32) + slot_base
    out = {}
    times = {}
    bn = tb.norm(dim=1)
    r = torch.empty_like(tb)
    stream = torch.cuda.current_stream()

    def timed(name, fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        x0, x, info = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        times[name] = e0.elapsed_time(e1) / 1000.0
        it, st, rr = kp.decode_info(info)
        assert (st == 0).all()
        ctx.residual(tops, tb, x0, r)
        out[name] = ((r.norm(dim=1) / bn).cpu().numpy(), it, x)

    def projected():
        x0 = torch.zeros_like(tgt_prev)
        ctx.project_targets_multi(n, slots, tops, tb, x0)       # paper: x0 = V H^-1 V^T b
        x = x0.clone()
        return x0, x, ctx.refine(tops, tb, x, tol=tol, m=m, maxit=1000)

    # pointer tables of the fixed target -> seed map, built once like a plan
    seed_rows = kp.ptrs([sx[int(k)] for k in group.target_seed])
    img_rows = kp.ptrs(img)
    xin = torch.empty((nt, 6, H * W), dtype=torch.float32, device=tgt_prev.device)
    delta = torch.empty((nt, 1, H * W), dtype=torch.float32, device=tgt_prev.device)

    def learned_():
        net.pack_inputs(img_rows, seed_rows, n / T, xin)
        for k in range(0, nt, net.max_batch):
            net.forward(xin[k:k + net.max_batch], delta[k:k + net.max_batch])
        x0 = torch.empty_like(tgt_prev)
        net.add_guess(delta, seed_rows, x0)                     # X_init = m_seed^n + Delta
        ctx.residual(tops, tb, x0, r)
        ctx.project_targets_multi(n, slots, tops, r, x0)        # + V H^-1 V^T (b - A X_init)
        x = x0.clone()
        return x0, x, ctx.refine(tops, tb, x, tol=tol, m=m, maxit=1000)

    def plain():
        x0 = torch.zeros_like(tgt_prev)
        x = x0.clone()
        return x0, x, ctx.refine(tops, tb, x, tol=tol, m=m, maxit=1000)

    timed("projected", projected)
    timed("learned", learned_)
    timed("plain", plain)
    out["times"] = times
    return out, sx
