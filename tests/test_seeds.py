"""Clustering-based seed choice (host logic): on images drawn from known
templates it recovers the templates, and its output is well formed."""
import numpy as np
import pytest

from paper_2511_17634_gb300 import seeds, synth


def test_recovers_the_templates_of_blob_images():
    # 30 targets of 3 templates (blob centres jittered by up to 2 px): every
    # chosen cluster is one template and every template gets one seed
    g = synth.make_group(321, 32, 32, 3, 3, 30)
    imgs = g.targets.reshape(30, 3, -1)                 # one row per image, all channels
    tmpl = np.arange(30) % 3
    sidx, assign = seeds.choose_seeds(imgs, 3, rng_seed=1)
    assert len(set(sidx.tolist())) == 3
    for j in range(3):
        assert len(set(tmpl[assign == j].tolist())) == 1
    assert sorted(tmpl[sidx].tolist()) == [0, 1, 2]


def test_seeds_belong_to_their_clusters_and_errors():
    rng = np.random.default_rng(0)
    X = rng.normal(size=(40, 7))
    sidx, assign = seeds.choose_seeds(X, 5, rng_seed=3)
    assert assign.shape == (40,) and set(assign.tolist()) <= set(range(5))
    assert all(assign[s] == j for j, s in enumerate(sidx))
    s2, a2 = seeds.choose_seeds(X, 5, rng_seed=3)
    assert np.array_equal(s2, sidx) and np.array_equal(a2, assign)   # deterministic
    with pytest.raises(ValueError):
        seeds.choose_seeds(X, 0)
    with pytest.raises(ValueError):
        seeds.choose_seeds(X, 41)


def test_ten_templates_one_seed_each():
    # the benchmark's shape (32x32x3, 10 templates): every template gets
    # exactly one seed and every cluster is one template
    g = synth.make_group(99, 32, 32, 3, 10, 100)
    imgs = g.targets.reshape(100, -1)
    tmpl = np.arange(100) % 10
    sidx, assign = seeds.choose_seeds(imgs, 10, rng_seed=0)
    assert sorted(tmpl[sidx].tolist()) == list(range(10))
    assert all(len(set(tmpl[assign == j].tolist())) == 1 for j in range(10))
