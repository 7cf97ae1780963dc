"""Choosing seed images for a set of targets (host-side preparation).

Sec. 3 solves one "seed" system per group of similar images and projects the
others onto its basis; the method assumes the seed resembles its targets.  For
a set of images whose groups are not known in advance, this picks k seeds by
k-means clustering of the images (k-means++ initialisation, Lloyd iterations)
and assigns every image to the seed of its cluster: the seed is the member
image closest to the cluster centre.  Plain numpy, deterministic for a given
generator seed; it runs once before a march, not on the solve path.
"""
from __future__ import annotations

import numpy as np


def _sq_dist(X, C):
    # ||x - c||^2 for all pairs, via ||x||^2 - 2 x.c + ||c||^2 (clamped at 0)
    d = (X * X).sum(1)[:, None] - 2.0 * X @ C.T + (C * C).sum(1)[None, :]
    return np.maximum(d, 0.0)


def _kmeans(X, k, iters, rng):
    n = X.shape[0]
    # k-means++: each next centre drawn with probability proportional to the
    # squared distance to the nearest centre chosen so far
    centres = [X[rng.integers(n)]]
    for _ in range(1, k):
        d = _sq_dist(X, np.array(centres)).min(1)
        tot = d.sum()
        p = d / tot if tot > 0 else np.full(n, 1.0 / n)
        centres.append(X[rng.choice(n, p=p)])
    C = np.array(centres)
    assign = np.full(n, -1)
    for _ in range(iters):
        new = _sq_dist(X, C).argmin(1)
        if np.array_equal(new, assign):
            break
        assign = new
        for j in range(k):
            members = X[assign == j]
            if len(members):
                C[j] = members.mean(0)
    inertia = _sq_dist(X, C)[np.arange(n), assign].sum()
    return C, assign, inertia


def choose_seeds(images, k, iters=50, rng_seed=0, restarts=8):
    """images: array [n][...] (one row per image, all channels together).
    Returns (seed_index [k] into images, assignment [n] in 0..k-1, the
    cluster of each image).  Every seed is assigned to its own cluster.  The
    clustering with the smallest within-cluster sum of squares over
    `restarts` k-means++ starts is kept (one start can settle in a local
    optimum that splits a group)."""
    X = np.asarray(images, dtype=np.float64).reshape(len(images), -1)
    n = X.shape[0]
    if not 1 <= k <= n:
        raise ValueError(f"need 1 <= k <= {n} seeds, got {k}")
    rng = np.random.default_rng(rng_seed)
    best = None
    for _ in range(max(1, restarts)):
        run = _kmeans(X, k, iters, rng)
        if best is None or run[2] < best[2]:
            best = run
    C, assign, _ = best
    # the seed of a cluster: its member closest to the centre (an empty
    # cluster takes the image farthest from every other centre)
    seeds = np.empty(k, dtype=np.int64)
    d = _sq_dist(X, C)
    taken = np.zeros(n, dtype=bool)
    for j in range(k):
        idx = np.flatnonzero(assign == j)
        if len(idx) == 0:
            cand = np.flatnonzero(~taken)
            idx = cand[[d[cand].min(1).argmax()]]
        best = idx[d[idx, j].argmin()]
        seeds[j] = best
        taken[best] = True
        assign[best] = j
    return seeds, assign
