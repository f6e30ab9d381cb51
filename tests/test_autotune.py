"""Autotuner host logic (CPU) and one tuning run on the GPU."""
import numpy as np
import pytest

from paper_2301_13601_gb300 import autotune, media


def test_chunk_candidates_bounds():
    c = autotune.chunk_candidates(8192, 4)
    assert c[0] == 0 and c[-1] == 8192
    assert all(h >= 64 for h in c[1:])
    assert autotune.chunk_candidates(40, 4) == [0, 40]


def test_pick_best_and_cache_round_trip(tmp_path, monkeypatch):
    monkeypatch.setenv(autotune.CACHE_ENV, str(tmp_path / "c.json"))
    cfg, sec = autotune.pick_best([({"k": 1}, 3.0), ({"k": 2}, 1.0), ({"k": 4}, 2.0)])
    assert cfg == {"k": 2} and sec == 1.0
    with pytest.raises(ValueError):
        autotune.pick_best([])
    autotune.save_cache({"a": {"steps_per_pass": 4}})
    assert autotune.load_cache() == {"a": {"steps_per_pass": 4}}


def test_missing_cache_is_empty(tmp_path, monkeypatch):
    monkeypatch.setenv(autotune.CACHE_ENV, str(tmp_path / "none" / "c.json"))
    assert autotune.load_cache() == {}


@pytest.mark.gpu
def test_tune_single_returns_a_working_config(tmp_path, monkeypatch):
    monkeypatch.setenv(autotune.CACHE_ENV, str(tmp_path / "c.json"))
    n = media.smooth_periodic_medium(512, 384, seed=1)
    best = autotune.tune_single(*n, 0.05, ks=(2, 4), steps=8, repeats=2)
    assert best["steps_per_pass"] in (2, 4) and best["chunk_rows"] in autotune.chunk_candidates(384, best["steps_per_pass"])
    assert best["site_updates_per_s"] > 0
    again = autotune.tune_single(*n, 0.05, ks=(2, 4), steps=8, repeats=2)
    assert again == best  # served from the cache


@pytest.mark.gpu
def test_batch_autotuner_in_the_loop(tmp_path, monkeypatch):
    """Batch(steps_per_pass=0) times the candidates, caches the choice and
    builds the batch with it; the result is the batch built with that choice
    explicitly, bit for bit."""
    from paper_2301_13601_gb300.qla import Batch

    monkeypatch.setenv(autotune.CACHE_ENV, str(tmp_path / "c.json"))
    rng = np.random.default_rng(9)
    inst = []
    for side, steps in ((256, 64), (384, 32), (512, 48)):
        w = media.random_ellipse_workload(rng, side, f"b{side}", 0.05, steps)
        inst.append({"n": w.medium(), "delta": w.delta, "nsteps": steps,
                     "pulse": ("Ez" if w.pulse.pol == media.POL_EZ else "Ey", w.pulse.x0, w.pulse.sigma, 1.0)})
    with Batch(inst, steps_per_pass=0) as b:
        tuned = dict(b.tuned)
        assert b.info()["steps_per_pass"] == tuned["steps_per_pass"] in (2, 4)
        b.run()
        auto = [b.get_fields(i) for i in range(len(inst))]
    assert autotune.load_cache()  # the choice was cached
    explicit = [dict(i, chunk_rows=tuned["chunk_rows"]) for i in inst]
    with Batch(explicit, steps_per_pass=tuned["steps_per_pass"]) as b:
        b.run()
        for i in range(len(inst)):
            assert np.array_equal(b.get_fields(i), auto[i])
    with Batch(inst, steps_per_pass=0) as b:  # served from the cache
        assert b.tuned == tuned
