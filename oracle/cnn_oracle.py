"""FP64 numpy reference of the learned-initial-guess network (not in the
paper): 3x3 convolutions with zero padding, ReLU between layers, MSE loss,
Adam.  TEST INFRASTRUCTURE ONLY -- used by tests/ to check the GPU forward
and backward kernels; it shares no code with them.

The network's kernels multiply BF16 operands with FP32 accumulation.  To
state their error bound rather than guess it, ``forward`` and
``loss_and_grads`` take an optional ``operand_round``: applied to exactly
the operands a BF16 tensor-core product would see -- every convolution's
input planes and weights in the forward pass; the output gradient, the
layer input and the weights in the two backward products -- while biases,
the bias gradient and every sum stay FP64.  ``bf16`` is that rounding
(nearest bfloat16, ties to even).  With it the reference differs from the
kernels only by FP32 accumulation; without it (the default) it is the
exact FP64 network.

Planes are arrays [batch][channel][W][H] (x index i first, y index j second,
the solver's vector order).  A layer's weights are [c_out][c_in][3][3] with
tap [di+1][dj+1] multiplying the input at (i+di, j+dj); the flat parameter
vector holds, per layer, the weights then the biases.
"""
import numpy as np


def unflatten(params, channels):
    out, o = [], 0
    for cin, cout in zip(channels[:-1], channels[1:]):
        w = params[o:o + cout * cin * 9].reshape(cout, cin, 3, 3)
        o += cout * cin * 9
        b = params[o:o + cout]
        o += cout
        out.append((w.astype(np.float64), b.astype(np.float64)))
    assert o == len(params)
    return out


def flatten(layers):
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in layers])


def bf16(a):
    """Round to the nearest bfloat16 (8 significant bits, ties to even), via
    float32 as a device conversion from an FP32 value does; returns float64."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + np.uint64(0x7FFF) + ((u >> np.uint64(16)) & np.uint64(1))) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64).reshape(np.shape(a))


def _ident(a):
    return a


def conv(x, w, b):
    """z[b,o,i,j] = b[o] + sum_{c,di,dj} w[o,c,di+1,dj+1] x[b,c,i+di,j+dj] (zero outside)."""
    B, C, W, H = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    z = np.zeros((B, w.shape[0], W, H)) + b[None, :, None, None]
    for di in (-1, 0, 1):
        for dj in (-1, 0, 1):
            z += np.einsum("oc,bcij->boij", w[:, :, di + 1, dj + 1],
                           xp[:, :, 1 + di:1 + di + W, 1 + dj:1 + dj + H])
    return z


def forward(params, channels, x, operand_round=None):
    """All layer outputs (post-activation; the last layer is linear).
    operand_round (e.g. ``bf16``) rounds each convolution's input planes and
    weights first."""
    rnd = operand_round or _ident
    acts = [x]
    layers = unflatten(params, channels)
    for k, (w, b) in enumerate(layers):
        z = conv(rnd(acts[-1]), rnd(w), b)
        acts.append(np.maximum(z, 0.0) if k + 1 < len(layers) else z)
    return acts


def loss_and_grads(params, channels, x, target, operand_round=None):
    """MSE over all outputs and its gradient with respect to every parameter.
    operand_round rounds the operands of the forward convolutions and of the
    two backward products (output gradient, layer input, weights)."""
    rnd = operand_round or _ident
    layers = unflatten(params, channels)
    acts = forward(params, channels, x, operand_round)
    out = acts[-1]
    n = out.size
    loss = float(np.mean((out - target) ** 2))
    dz = 2.0 * (out - target) / n
    grads = []
    for k in range(len(layers) - 1, -1, -1):
        w, b = layers[k]
        xin = acts[k]
        B, C, W, H = xin.shape
        xp = np.pad(rnd(xin), ((0, 0), (0, 0), (1, 1), (1, 1)))
        dzr = rnd(dz)
        dw = np.zeros_like(w)
        for di in (-1, 0, 1):
            for dj in (-1, 0, 1):
                dw[:, :, di + 1, dj + 1] = np.einsum("boij,bcij->oc", dzr,
                                                     xp[:, :, 1 + di:1 + di + W, 1 + dj:1 + dj + H])
        db = dz.sum(axis=(0, 2, 3))
        grads.append((dw, db))
        if k == 0:
            break
        dzp = np.pad(dzr, ((0, 0), (0, 0), (1, 1), (1, 1)))
        wr = rnd(w)
        dx = np.zeros_like(xin)
        for di in (-1, 0, 1):
            for dj in (-1, 0, 1):
                dx += np.einsum("oc,boij->bcij", wr[:, :, di + 1, dj + 1],
                                dzp[:, :, 1 - di:1 - di + W, 1 - dj:1 - dj + H])
        dz = dx * (acts[k] > 0)                  # through the previous ReLU
    return loss, flatten(grads[::-1])


def adam(params, grads, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015); returns (params, m, v)."""
    m = b1 * m + (1 - b1) * grads
    v = b2 * v + (1 - b2) * grads * grads
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


# ---------------------------------------------------------------------------
# The learned initial guess of a target solve at timestep n (not in the
# paper; the workload's learned-guess configuration).  Reading of "inputs =
# target image + seed solution at timestep t + t embedding": the target image
# as the march has carried it to timestep n-1 (its lagged field m_i^{n-1};
# the image itself at n = 1), the seed's solution m_seed^n of the same
# timestep, four time planes tau, 1 - tau, sin(pi tau), cos(pi tau) for
# tau = n / T (each distinct over 0 < tau <= 1), and, derived from the
# target image and t, the residual the step leaves at the image,
# r = m^{n-1}/dt - A m^{n-1} (A of Sec. 2.3 at timestep n, lagged on m^{n-1}),
# scaled to unit rms: r_hat = r / rho, rho = ||r|| / sqrt(N).  The step's
# change solves A (m^n - m^{n-1}) = r, so in units of dt rho it is the
# near-identity local operator (dt A)^{-1} applied to r_hat -- of order one
# at every timestep, although rho falls by orders of magnitude over the
# march as the images smooth.  The guess is
#     x_init = m_i^{n-1} + dt rho * net(...).
#
# The fields enter as two planes each, hi = bf16(v) and lo = 256 (v - hi):
# one BF16 plane carries 8 significant bits (an absolute 2e-3 at m = 0.5),
# and the step's change is a difference of neighbouring values a few hundred
# times smaller than m, so one plane would bury it in rounding; the pair
# carries about 16 bits and the first layer's products recombine it.

NIN = 10       # input planes of the learned guess


def split_hi_lo(m):
    """(hi, lo) with hi = bf16(m), lo = 256 (m - hi); m = hi + lo / 256."""
    m = np.asarray(m, dtype=np.float64)
    hi = bf16(m)
    return hi, 256.0 * (m - hi)


def step_residual(mprev, g2n, T, H, W):
    """r = m/dt - A(m~ = m) m per channel (Sec. 2.3, f = 0) and rho =
    ||r|| / sqrt(N); rows of mprev are channels in the solver order."""
    from . import oracle as O
    mprev = np.asarray(mprev, dtype=np.float64)
    dt, h = 1.0 / T, 1.0 / H
    r = np.empty_like(mprev)
    for k in range(mprev.shape[0]):
        C = O.coeffs(H, W, g2n, dt, h, mprev[k])
        r[k] = O.rhs(H, W, dt, h, mprev[k]) - O.apply(H, W, C, mprev[k])
    rho = np.sqrt(np.mean(r * r, axis=1))
    return r, rho


def network_inputs(mprev, mseed, n, T, g2n, H, W):
    """Planes [B][10][N]: m_i^{n-1} (hi, lo), m_seed^n (hi, lo), tau, 1 - tau,
    sin pi tau, cos pi tau with tau = n / T (n = 1..T), r_hat (hi, lo); and
    rho per channel (see step_residual)."""
    mprev = np.asarray(mprev, dtype=np.float64)
    B, N = mprev.shape
    tau = n / T
    r, rho = step_residual(mprev, g2n, T, H, W)
    rhat = np.where(rho[:, None] > 0, r / np.where(rho > 0, rho, 1.0)[:, None], 0.0)
    out = np.empty((B, NIN, N))
    out[:, 0], out[:, 1] = split_hi_lo(mprev)
    out[:, 2], out[:, 3] = split_hi_lo(np.asarray(mseed, dtype=np.float64).reshape(B, N))
    for k, v in enumerate((tau, 1.0 - tau, np.sin(np.pi * tau), np.cos(np.pi * tau))):
        out[:, 4 + k] = v
    out[:, 8], out[:, 9] = split_hi_lo(rhat)
    return out, rho


def learned_guess(params, channels, mprev, mseed, n, T, g2n, H, W, operand_round=None):
    """x_init = m_i^{n-1} + dt rho * net([m_i^{n-1}, m_seed^n, time planes,
    r_hat]) for a batch of target channels ([B][N] arrays, N = H*W in the
    solver order)."""
    mprev = np.asarray(mprev, dtype=np.float64)
    B, N = mprev.shape
    x, rho = network_inputs(mprev, mseed, n, T, g2n, H, W)
    d = forward(params, channels, x.reshape(B, NIN, W, H), operand_round)[-1].reshape(B, N)
    return mprev + (1.0 / T) * rho[:, None] * d
