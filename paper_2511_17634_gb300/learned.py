"""Learned initial guess for the target solves (not in the paper).

A small 3x3 convolutional network (kp.CNN, trained with the library's own
tensor-core kernels) maps [m_i^{n-1}, m_seed^n, time embedding, r_hat] --
the target's image as the march has carried it to timestep n-1, the seed's
solution of timestep n, tau = n/T, 1 - tau, sin(pi tau), cos(pi tau), and
the residual the step leaves at the image, r = m^{n-1}/dt - A m^{n-1}, over
its rms rho (the fields each as a hi and a lo BF16 plane) -- to the step's
change in units of dt rho.  The step's change solves A (m^n - m^{n-1}) = r,
so in those units it is the near-identity operator (dt A)^{-1} applied to
r_hat, of order one at every timestep although rho falls by orders of
magnitude as the images smooth.  The target's initial guess is

    x_init = m_i^{n-1} + dt rho * net(...),

judged against the warm start m_i^{n-1} by FP64 residual norm, projected in
residual form onto the seed's Krylov basis when kept (x0 = x_init + V_a
H_a^{-1} V_a^T (b - A x_init), Sec. 3 Phase 2), and refined by GMRES to the
same tolerance as every other solve, so the network changes the cost of a
solve, never its accuracy.  In the time march (kp.MARCH_LEARNED) all of it
runs on the GPU inside the march's per-timestep graph.

Host orchestration only (pair generation, the training loop, timing of the
march modes): every arithmetic step runs in the CUDA library.
"""
from __future__ import annotations

import numpy as np

from . import kp

# the workload's network: four 3x3 layers, 32 hidden channels.  A narrower
# one (channels=(10, 16, 16, 1)) leaves about the same GMRES steps per solve
# (4.51 against 4.48 at 128x128x3) at 0.6x the inference time -- the layers
# are bound by the HBM traffic of their activations
CHANNELS = (10, 32, 32, 32, 1)


def init_params(seed=0, channels=CHANNELS):
    """He-style initial weights, zero biases, in the network's flat layout;
    the last layer starts near zero, so x_init starts at the warm start."""
    rng = np.random.default_rng(seed)
    parts = []
    for ci, co in zip(channels[:-1], channels[1:]):
        parts.append(rng.normal(scale=np.sqrt(2.0 / (9 * ci)), size=co * ci * 9))
        parts.append(np.zeros(co))
    p = np.concatenate(parts)
    nlast = channels[-2] * 9 * channels[-1]
    p[-(nlast + channels[-1]):-channels[-1]] *= 0.01
    return p.astype(np.float32)


def generate_pairs(ctx, net, group, T, g2, steps, every, tol_seed=1e-10, tol=1e-8, m=40,
                   mode=kp.MARCH_PROJECTED):
    """Run the method (a march of the group's seeds and targets) over
    `steps` timesteps and, at every `every`-th timestep n, record the network
    input [m_i^{n-1} (hi, lo), m_seed^n (hi, lo), time planes, r_hat (hi, lo)]
    and the training target (m_i^n - m_i^{n-1}) / (dt rho) of every target
    channel.  Returns float32 CUDA tensors (inputs [pairs][10][P], targets
    [pairs][1][P])."""
    import torch
    H, W = group.H, group.W
    P = H * W
    dev = torch.device("cuda", torch.cuda.current_device())
    s = torch.as_tensor(group.seeds.reshape(len(group.seeds), -1).copy(), device=dev)
    t = torch.as_tensor(group.targets.reshape(len(group.targets), -1).copy(), device=dev)
    plan = kp.March(ctx, [(s, t, group.target_seed, H, W)], T, g2, mode=mode, tol_seed=tol_seed, tol=tol,
                    m_seed=m, m=m)
    ins, outs = [], []
    nt = t.shape[0]
    done = 0
    for n in range(every, steps + 1, every):
        plan.run(done, n - 1 - done)
        prev = t.clone()
        plan.run(n - 1, 1)
        done = n
        seed_rows = [s[int(k)] for k in group.target_seed]
        x = torch.empty((nt, CHANNELS[0], P), dtype=torch.float32, device=dev)
        y = torch.empty((nt, 1, P), dtype=torch.float32, device=dev)
        rho = torch.empty(nt, dtype=torch.float64, device=dev)
        net.pack_inputs(prev, seed_rows, n, T, float(g2[n - 1]), x, rho)
        net.pack_target(t, prev, y, scale=float(T), rho=rho)        # (m^n - m^{n-1}) / (dt rho)
        ins.append(x)
        outs.append(y)
    plan.close()
    torch.cuda.synchronize()
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


def compare_modes(ctx, net, seeds, targets, target_seed, H, W, T, g2, n0, steps, modes, tol_seed=1e-10,
                  tol=1e-8, m=40):
    """From the states (seeds, targets: CUDA (k, N) float64 at timestep n0)
    march timesteps n0+1 .. n0+steps in each of `modes` ({name: kp march
    mode}) and return {name: (final targets, step stats, timing)}; every run
    starts from the same states."""
    out = {}
    for name, mode in modes.items():
        s, t = seeds.clone(), targets.clone()
        plan = kp.March(ctx, [(s, t, target_seed, H, W)], T, g2, mode=mode, tol_seed=tol_seed, tol=tol,
                        m_seed=m, m=m, cnn=net if mode in (kp.MARCH_LEARNED, kp.MARCH_LEARNED_ONLY) else None)
        st, tm = plan.run(n0, steps, stats=True, timing=True)
        out[name] = (t, st, tm)
        plan.close()
    return out
