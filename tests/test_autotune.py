"""Autotuner: cache keys and persistence (CPU), and tuned filters on the GPU."""
import json
import os

import numpy as np
import pytest

import synthetic as S


def test_cache_roundtrip_and_best_pick(tmp_path, monkeypatch):
    from paper_1812_01502_gb300 import autotune
    path = str(tmp_path / "tune.json")
    monkeypatch.setenv("BFPF_TUNE_CACHE", path)
    k = autotune.problem_key("NVIDIA GB300", 152, "sv", 1, 1 << 24, (16,) * 6)
    assert k == "NVIDIA GB300|152|sv|d1|N16777216|r16x16x16x16x16x16"
    autotune.store(k, {"tile": 2048, "grid": 152, "ms_per_step": 0.08})
    autotune.store("other", {"tile": 0, "grid": 0, "ms_per_step": 1.0})
    data = autotune.load_cache()
    assert data[k]["tile"] == 2048 and "other" in data
    assert json.load(open(path))[k]["grid"] == 152
    best, ms = autotune.pick_best({(0, 0): 0.09, (1024, 152): 0.07, (2048, 304): 0.08})
    assert best == (1024, 152) and ms == 0.07
    cands = list(autotune.candidates(152, 1))
    assert (0, 0) in cands and len(cands) == len(set(cands))


def test_missing_or_corrupt_cache_is_empty(tmp_path, monkeypatch):
    from paper_1812_01502_gb300 import autotune
    p = tmp_path / "bad.json"
    p.write_text("{not json")
    monkeypatch.setenv("BFPF_TUNE_CACHE", str(p))
    assert autotune.load_cache() == {}
    monkeypatch.setenv("BFPF_TUNE_CACHE", str(tmp_path / "absent.json"))
    assert autotune.load_cache() == {}


@pytest.mark.gpu
def test_tuned_filter_matches_default(bfpf, tmp_path, monkeypatch):
    monkeypatch.setenv("BFPF_TUNE_CACHE", str(tmp_path / "tune.json"))
    from paper_1812_01502_gb300 import autotune
    model = S.lg_dense(2, seed=5)
    radices = (3, 5, 16, 8)                 # tile-kernel digits (3, 5) and group-kernel digits
    N = int(np.prod(radices))
    entry = autotune.tune(model, N, radices)
    assert entry["ms_per_step"] <= entry["default_ms_per_step"] + 1e-9
    assert autotune.tune(model, N, radices) == entry        # served from the cache
    y = S.simulate(model, 12, seed=1)[1]
    a = bfpf.ButterflyFilter(model, N, radices, 3, tune=True)
    b = bfpf.ButterflyFilter(model, N, radices, 3)
    ra, rb = a.run(y), b.run(y)
    # the first increment depends only on pi_0 and y_0 (identical draws); later steps may
    # differ by a rare draw flip because the grid changes the partial-sum order of mu
    np.testing.assert_allclose(ra["inc"][:1], rb["inc"][:1], rtol=1e-6, atol=1e-6)
    assert np.all(np.isfinite(ra["inc"]))
    a.close()
    b.close()
