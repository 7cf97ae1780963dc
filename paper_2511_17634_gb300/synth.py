"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds input generation only (images, the g^2 schedule, the
seed/target assignment); none of the solver's arithmetic lives here.  The
CUDA path, the benchmark and the CPU oracle all draw their inputs from it.

The paper measures on CIFAR-10 (32x32) and CelebA (64x64, 128x128) images
(Sec. 5, Table 4).  Neither dataset is used: these blob images stand in for
them with the same shapes.  Each channel is

    clip( clip(sum of 6 axis-aligned Gaussian blobs, 0, 1) + N(0, 0.02^2), 0, 1 )

with blob centres uniform on the grid, widths sigma_x, sigma_y ~ U(1.5, 4) px,
amplitudes ~ U(0.3, 1) drawn per channel (centres shared by the channels of
one image).  A seed image uses its template's centres exactly; a target image
uses the template's centres jittered by U(-2, 2) px per coordinate and draws
its own widths, amplitudes and noise.

Random numbers come from a counter-based generator (SplitMix64 finaliser of
key + counter, Steele et al. 2014) so that every value depends only on
(seed, stream, index) and is identical on every host and numpy version.

Layout: a channel is an array of shape (W, H), C order, i.e. index i*H + j
with i the x (column) and j the y (row) coordinate -- the y-fastest order of
Sec. 2.3, Eq. (14).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLD = np.uint64(0x9E3779B97F4A7C15)


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def _key(*parts: int) -> np.uint64:
    k = np.uint64(0x2545F4914F6CDD1D)
    with np.errstate(over="ignore"):
        for p in parts:
            k = _mix(np.array([k ^ (np.uint64(p & 0xFFFFFFFFFFFFFFFF) * _GOLD)],
                              dtype=np.uint64))[0]
    return k


def uniform(key: np.uint64, n: int, offset: int = 0) -> np.ndarray:
    """n uniforms in [0, 1) from stream `key`, counters offset..offset+n-1."""
    ctr = np.arange(offset, offset + n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _mix(key + (ctr + np.uint64(1)) * _GOLD)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(key: np.uint64, n: int) -> np.ndarray:
    """n standard normals by Box-Muller on pairs of uniforms."""
    m = (n + 1) // 2
    u1 = uniform(key, m, 0)
    u2 = uniform(key, m, m)
    r = np.sqrt(-2.0 * np.log1p(-u1))          # 1-u1 in (0, 1]
    z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])
    return z[:n]


NBLOBS = 6


def template_centres(seed: int, template: int, H: int, W: int) -> np.ndarray:
    """(NBLOBS, 2) blob centres (x in [0,W), y in [0,H)) of one template."""
    u = uniform(_key(seed, 1, template), 2 * NBLOBS)
    return np.stack([u[0::2] * W, u[1::2] * H], axis=1)


def blob_image(H: int, W: int, channels: int, centres: np.ndarray, key: np.uint64,
               noise: float = 0.02) -> np.ndarray:
    """One image, shape (channels, W, H), values in [0, 1]."""
    u = uniform(key, 2 * NBLOBS + channels * NBLOBS)
    sx = 1.5 + 2.5 * u[0:NBLOBS]
    sy = 1.5 + 2.5 * u[NBLOBS:2 * NBLOBS]
    amp = 0.3 + 0.7 * u[2 * NBLOBS:].reshape(channels, NBLOBS)
    x = np.arange(W, dtype=np.float64)[:, None]
    y = np.arange(H, dtype=np.float64)[None, :]
    out = np.zeros((channels, W, H))
    z = normal(_key(int(key), 7), channels * W * H).reshape(channels, W, H)
    for c in range(channels):
        img = np.zeros((W, H))
        for b in range(NBLOBS):
            img += amp[c, b] * np.exp(-((x - centres[b, 0]) ** 2) / (2 * sx[b] ** 2)
                                      - ((y - centres[b, 1]) ** 2) / (2 * sy[b] ** 2))
        out[c] = np.clip(np.clip(img, 0.0, 1.0) + noise * z[c], 0.0, 1.0)
    return out


def beta_schedule(T: int, beta_min: float = 1e-4, beta_max: float = 0.02) -> np.ndarray:
    """(g^n)^2 for n = 1..T: linear from beta_min to beta_max (DDPM-style
    linear schedule).  The paper's own experiments use constant g = 0.5
    (Sec. 5), available as ``constant_g2(T, 0.5)``."""
    if T == 1:
        return np.array([beta_min])
    n = np.arange(T, dtype=np.float64)
    return beta_min + n * (beta_max - beta_min) / (T - 1)


def constant_g2(T: int, g: float = 0.5) -> np.ndarray:
    return np.full(T, g * g)


@dataclass
class Group:
    """Seed and target channels of one grid size.

    seeds: (n_seed_planes, W, H); targets: (n_target_planes, W, H);
    target_seed[k] = index of the seed plane serving target plane k.
    """
    H: int
    W: int
    seeds: np.ndarray
    targets: np.ndarray
    target_seed: np.ndarray
    channels: int = 1

    @property
    def N(self) -> int:
        return self.H * self.W


@dataclass
class Workload:
    name: str
    T: int
    g2: np.ndarray
    groups: list = field(default_factory=list)
    tol_seed: float = 1e-10
    tol: float = 1e-8
    m_seed: int = 40
    m: int = 40
    a: int = 40
    precision: str = "fp64"

    @property
    def n_target_planes(self) -> int:
        return sum(g.targets.shape[0] for g in self.groups)

    @property
    def n_seed_planes(self) -> int:
        return sum(g.seeds.shape[0] for g in self.groups)


def make_group(seed: int, H: int, W: int, channels: int, ntemplates: int, ntargets: int,
               jitter: float = 2.0, tag: int = 0, target_offset: int = 0) -> Group:
    """Seeds = one image per template; targets cycle over the templates
    (target t uses template t mod ntemplates)."""
    cent = [template_centres(seed + 1000 * tag, k, H, W) for k in range(ntemplates)]
    seeds = np.concatenate([blob_image(H, W, channels, cent[k], _key(seed, tag, 2, k))
                            for k in range(ntemplates)])
    tg, ts = [], []
    for t in range(target_offset, target_offset + ntargets):
        k = t % ntemplates
        ju = uniform(_key(seed, tag, 3, t), 2 * NBLOBS).reshape(NBLOBS, 2)
        c = cent[k] + jitter * (2.0 * ju - 1.0)
        tg.append(blob_image(H, W, channels, c, _key(seed, tag, 4, t)))
        ts.extend(k * channels + ch for ch in range(channels))
    targets = np.concatenate(tg) if tg else np.zeros((0, W, H))
    return Group(H=H, W=W, seeds=seeds, targets=targets,
                 target_seed=np.array(ts, dtype=np.int32), channels=channels)


def config(idx: int, seed: int | None = None, T: int | None = None,
           ntargets: int | None = None) -> Workload:
    """The five workloads (index 1..5), optionally with fewer timesteps or
    targets for tests.  Generator seed defaults to 1234 + idx."""
    s = 1234 + idx if seed is None else seed
    if idx == 1:     # 1 seed + 4 targets, 28x28x1, T=50, GMRES(30), seed tol 1e-10
        TT = T or 50
        g = [make_group(s, 28, 28, 1, 1, ntargets or 4)]
        return Workload("tiny-28x28x1", TT, beta_schedule(TT), g, m_seed=30, m=30, a=30)
    if idx == 2:     # 10 templates, 256 targets, 32x32x3, T=1000, m=40, FP64
        TT = T or 1000
        g = [make_group(s, 32, 32, 3, 10, ntargets or 256)]
        return Workload("blobs-32x32x3-10seeds-256targets", TT, beta_schedule(TT), g)
    if idx == 3:     # 2048 targets over three sizes, 16 seeds, T=1000
        TT = T or 1000
        nt = ntargets or 2048
        sizes = [(28, 28, 1, 6), (32, 32, 3, 5), (64, 64, 3, 5)]
        per = [nt // 3 + (1 if k < nt % 3 else 0) for k in range(3)]
        g = [make_group(s, H, W, C, nk, per[k], tag=k + 1)
             for k, (H, W, C, nk) in enumerate(sizes)]
        return Workload("mixed-28-32-64-16seeds-2048targets", TT, beta_schedule(TT), g)
    if idx == 4:     # 64x64x3, 8 seeds + 1024 targets, mixed precision
        TT = T or 1000
        g = [make_group(s, 64, 64, 3, 8, ntargets or 1024)]
        return Workload("blobs-64x64x3-8seeds-1024targets", TT, beta_schedule(TT), g,
                        precision="mixed")
    if idx == 5:     # 128x128x3, 16 seeds + 4096 targets, learned guess
        TT = T or 1000
        g = [make_group(s, 128, 128, 3, 16, ntargets or 4096)]
        return Workload("blobs-128x128x3-16seeds-4096targets", TT, beta_schedule(TT), g,
                        precision="mixed")
    raise ValueError(f"unknown workload {idx}")
