"""FP64 numpy reference of the learned-initial-guess network (not in the
paper): 3x3 convolutions with zero padding, ReLU between layers, MSE loss,
Adam.  TEST INFRASTRUCTURE ONLY -- used by tests/ to check the GPU forward
and backward kernels; it shares no code with them.

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


def forward(params, channels, x):
    """All layer outputs (post-activation; the last layer is linear)."""
    acts = [x]
    layers = unflatten(params, channels)
    for k, (w, b) in enumerate(layers):
        z = conv(acts[-1], w, b)
        acts.append(np.maximum(z, 0.0) if k + 1 < len(layers) else z)
    return acts


def loss_and_grads(params, channels, x, target):
    """MSE over all outputs and its gradient with respect to every parameter."""
    layers = unflatten(params, channels)
    acts = forward(params, channels, x)
    out = acts[-1]
    n = out.size
    loss = float(np.mean((out - target) ** 2))
    dz = 2.0 * (out - target) / n
    grads = []
    for k in range(len(layers) - 1, -1, -1):
        w, b = layers[k]
        xin = acts[k]
        B, C, W, H = xin.shape
        xp = np.pad(xin, ((0, 0), (0, 0), (1, 1), (1, 1)))
        dw = np.zeros_like(w)
        for di in (-1, 0, 1):
            for dj in (-1, 0, 1):
                dw[:, :, di + 1, dj + 1] = np.einsum("boij,bcij->oc", dz,
                                                     xp[:, :, 1 + di:1 + di + W, 1 + dj:1 + dj + H])
        db = dz.sum(axis=(0, 2, 3))
        grads.append((dw, db))
        if k == 0:
            break
        dzp = np.pad(dz, ((0, 0), (0, 0), (1, 1), (1, 1)))
        dx = np.zeros_like(xin)
        for di in (-1, 0, 1):
            for dj in (-1, 0, 1):
                dx += np.einsum("oc,boij->bcij", w[:, :, di + 1, dj + 1],
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
