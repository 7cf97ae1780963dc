"""Host logic of the autotuner: candidate choice and the JSON cache; one GPU
run over every candidate."""
import pytest

from paper_2511_17634_gb300 import autotune, synth


def test_choose_prefers_fastest_then_smaller_m():
    t = {(20, 0, (256, 2)): 2.0, (30, 0, (256, 2)): 1.0, (40, 0, (128, 4)): 1.0,
         (60, 6, (256, 2)): 3.0}
    assert autotune.choose(t) == (30, 0, (256, 2))


def test_tune_times_every_candidate_and_caches(tmp_path):
    wl = synth.config(1, T=4)
    calls = []

    def fake(m, S, shape):
        calls.append((m, S, shape))
        return abs(m - 40) + 0.1 * S + (0.0 if shape == (128, 4) else 0.01)

    path = str(tmp_path / "tune.json")
    r = autotune.tune(wl, cache_path=path, time_fn=fake)
    assert r["m"] == 40 and r["smem_vectors"] == 0
    assert (r["block_threads"], r["blocks_per_sm"]) == (128, 4)
    assert len(calls) == (len(autotune.M_CANDIDATES) * len(autotune.WINDOW_CANDIDATES)
                          * len(autotune.SHAPE_CANDIDATES))
    r2 = autotune.tune(wl, cache_path=path, time_fn=lambda m, S, nt: 1 / 0)   # from the cache
    assert r2["m"] == 40


@pytest.mark.gpu
def test_tune_on_gpu_picks_a_candidate(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_17634_gb300 import build
    build.build()
    wl = synth.config(2, T=1000, ntargets=16)
    r = autotune.tune(wl, steps=2, cache_path=str(tmp_path / "t.json"))
    assert r["m"] in autotune.M_CANDIDATES and r["smem_vectors"] in autotune.WINDOW_CANDIDATES
    assert len(r["timings"]) == (len(autotune.M_CANDIDATES) * len(autotune.WINDOW_CANDIDATES)
                                 * len(autotune.SHAPE_CANDIDATES))


