"""Host logic of the autotuner: candidate choice and the JSON cache."""
from paper_2511_17634_gb300 import autotune, synth


def test_choose_prefers_fastest_then_smaller_m():
    t = {(20, 0): 2.0, (30, 0): 1.0, (40, 0): 1.0, (60, 6): 3.0}
    assert autotune.choose(t) == (30, 0)


def test_tune_times_every_candidate_and_caches(tmp_path):
    wl = synth.config(1, T=4)
    calls = []

    def fake(m, S):
        calls.append((m, S))
        return abs(m - 40) + 0.1 * S

    path = str(tmp_path / "tune.json")
    r = autotune.tune(wl, cache_path=path, time_fn=fake)
    assert r["m"] == 40 and r["smem_vectors"] == 0
    assert len(calls) == len(autotune.M_CANDIDATES) * len(autotune.WINDOW_CANDIDATES)
    r2 = autotune.tune(wl, cache_path=path, time_fn=lambda m, S: 1 / 0)   # served from the cache
    assert r2["m"] == 40
