"""Host logic of the launch-shape autotuner: cache key, cache round trip and
the cached answer returned without touching a GPU."""
import json

import torch

from paper_2208_14961_gb300 import autotune


def test_cached_choice_is_returned_without_a_gpu(tmp_path, monkeypatch):
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "autotune.json"))
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a, **k: "NVIDIA GB300")
    specs = [(12, 4644), (36, 3175)]
    key = autotune._key(specs)
    assert key == "NVIDIA_GB300|m12P18576,m36P12700"
    autotune._save({key: {"blocks": 114, "ms_per_generation": {"114": 0.05}}})
    assert json.load(open(autotune.CACHE))[key]["blocks"] == 114
    assert autotune.tune_fused_grid(specs) == 114
    # a cached shape is returned as stored
    skey = "NVIDIA_GB300|shape|m36P12700"
    autotune._save({skey: {"tpp": 0, "nch": 5, "ms_per_generation": {}}})
    assert autotune.tune_shape(36, 3175) == {"tpp": 0, "nch": 5, "ms_per_generation": {}}


def test_missing_or_broken_cache_reads_as_empty(tmp_path, monkeypatch):
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "none.json"))
    assert autotune._load() == {}
    p = tmp_path / "bad.json"
    p.write_text("{not json")
    monkeypatch.setattr(autotune, "CACHE", str(p))
    assert autotune._load() == {}


def test_shape_candidates_include_the_built_in_choice():
    """m <= 32: two and four threads per pair; m > 32: chunkings up to
    min(16, m/2), always including the library's own cost-model choice
    (m = 100: costs rounds * (run + 2) = 208, 189, 190, 195, 192 for 1..5
    chunks, so 2)."""
    assert autotune.shape_candidates(20) == [(4, 0), (2, 0)]
    for m in (36, 64, 100, 128):
        c = autotune.shape_candidates(m)
        assert (0, autotune.warp_gram_chunks(m)) in c
        assert all(1 <= n <= min(16, m // 2) and t == 0 for t, n in c)
    assert autotune.warp_gram_chunks(100) == 2
