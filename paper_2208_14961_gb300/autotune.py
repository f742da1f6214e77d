"""Autotuner of the persistent generation kernel's launch shape.

The fused kernel is latency bound (two grid barriers per generation); the
number of resident blocks trades build parallelism against barrier and
per-block scan cost.  For a set of populations (their orders and sizes) the
tuner times a few generations of throw-away copies at each candidate block
count, picks the fastest and caches the choice in a JSON file keyed by GPU
name and population shapes.
"""
from __future__ import annotations

import json
import os

import torch

from . import hadga as h

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


def _key(specs):
    name = torch.cuda.get_device_name().replace(" ", "_")
    return name + "|" + ",".join(f"m{m}P{4 * N}" for m, N in specs)


def _load():
    try:
        with open(CACHE) as fh:
            return json.load(fh)
    except Exception:
        return {}


def _save(d):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(d, fh, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def tune_fused_grid(specs, generations: int = 32, stream=None, use_cache: bool = True) -> int:
    """specs: list of (m, N).  Returns the chosen block count (0 = all SMs)."""
    key = _key(specs)
    cache = _load() if use_cache else {}
    if key in cache:
        return int(cache[key]["blocks"])
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    candidates = sorted({max(1, sms // 4), sms // 2, (3 * sms) // 4, sms})
    stream = stream if stream is not None else torch.cuda.Stream()
    pops = []
    for idx, (m, N) in enumerate(specs):
        p = h.Population(m, N, seed=12345, pop_id=idx, storage=h.STORE_BITS, traj_cap=generations, stream=stream)
        p.init_population()
        p.fitness()
        pops.append(p)
    times = {}
    for b in candidates:
        h.set_fused_grid(pops[0], b)
        h.step_multi(pops, 4)  # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h.step_multi(pops, generations)
        e1.record(stream)
        e1.synchronize()
        times[b] = e0.elapsed_time(e1)
    for p in pops:
        p.close()
    best = min(times, key=times.get)
    cache[key] = {"blocks": int(best), "ms_per_generation": {str(k): v / generations for k, v in times.items()}}
    if use_cache:
        _save(cache)
    return int(best)
