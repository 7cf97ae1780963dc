"""Writes tiny_march.json: the oracle's states after a few timesteps of the
tiny 28x28 workload, at sampled grid points.  Calls only the oracle."""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import oracle as O  # noqa: E402
from paper_2511_17634_gb300 import synth  # noqa: E402

STEPS = 5
SAMPLES = [0, 1, 27, 28, 391, 392, 500, 783]


def record():
    wl = synth.config(1)
    g = wl.groups[0]
    ms, mt, st = O.march(g.H, g.W, wl.T, wl.g2, g.seeds, g.targets, g.target_seed, steps=STEPS,
                         tol_seed=1e-12, m_seed=30, a=30, tol_ref=1e-12, m_ref=30)
    return {
        "workload": wl.name, "steps": STEPS, "tol": 1e-12, "samples": SAMPLES,
        "seed": [float(ms[0][k]) for k in SAMPLES],
        "targets": [[float(mt[t][k]) for k in SAMPLES] for t in range(len(mt))],
        "seed_iters": [int(s.seed_iters[0]) for s in st],
    }


if __name__ == "__main__":
    with open(os.path.join(HERE, "tiny_march.json"), "w") as f:
        json.dump(record(), f, indent=1)
