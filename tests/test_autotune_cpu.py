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


def test_missing_or_broken_cache_reads_as_empty(tmp_path, monkeypatch):
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "none.json"))
    assert autotune._load() == {}
    p = tmp_path / "bad.json"
    p.write_text("{not json")
    monkeypatch.setattr(autotune, "CACHE", str(p))
    assert autotune._load() == {}
