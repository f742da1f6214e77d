"""Autotuner of the persistent generation kernel and of the Gram path.

Choices are measured on the GPU at hand and cached in a JSON file keyed by
GPU name and shape; every choice gives bit-identical results, only speed
differs.

* Launch shape per order m (`tune_shape`): threads per pair of the m <= 32
  build (2: a thread computes a whole offspring; 4: a thread computes half
  of its fitness terms) or the warp-Gram work split of m > 32 (chunks per
  column, i.e. how the m(m-1)/2 column pairs spread over a warp's lanes).
  Candidates are timed in alternation on one population, twice each.
* Block count of a launch over a set of populations (`tune_fused`), with
  the populations' tuned shapes applied.
* Gram path per (storage, m, fitness kind) for GA_PATH_AUTO
  (`tune_gram_path`): every exact path the library accepts is timed on a
  population of about 2 GiB (int8 size; well beyond the L2, where the
  paths' HBM and tail behaviour match large workloads: a quarter GiB picked
  the tcgen05 path at m = 64, which is slower than the warp-level FP8 MMA at
  8 GiB) and the fastest is set as the process-wide AUTO choice
  (ga_set_auto_path).
"""
from __future__ import annotations

import json
import os

import torch

from . import hadga as h

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


def _gpu():
    return torch.cuda.get_device_name().replace(" ", "_")


def _key(specs):
    return _gpu() + "|" + ",".join(f"m{m}P{4 * N}" for m, N in specs)


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


def warp_gram_chunks(m: int) -> int:
    """The library's built-in chunks per column (its cost model), so that the
    tuner always measures the default next to the alternatives."""
    half = m >> 1
    best, best_cost = 1, 1 << 30
    for n in range(1, min(16, half) + 1):
        rounds = (m * n + 31) >> 5
        run = (half + n - 1) // n
        cost = rounds * (run + 2)
        if cost < best_cost:
            best, best_cost = n, cost
    return best


def shape_candidates(m: int):
    """(tpp, nch) pairs measured for order m."""
    if m <= 32:
        return [(4, 0), (2, 0)]
    top = min(16, m // 2)
    nchs = sorted({n for n in (1, 2, 3, 4, 6, 8, 12, 16) if n <= top} | {warp_gram_chunks(m)})
    return [(0, n) for n in nchs]


def _time(pops, generations, stream):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    h.step_multi(pops, generations)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1)


def tune_shape(m: int, N: int, generations: int = 32, stream=None, use_cache: bool = True) -> dict:
    """Launch shape of order m at population size 4N: {"tpp", "nch",
    "ms_per_generation": {candidate: ms}}."""
    key = f"{_gpu()}|shape|m{m}P{4 * N}"
    cache = _load() if use_cache else {}
    if key in cache:
        return cache[key]
    stream = stream if stream is not None else torch.cuda.Stream()
    p = h.Population(m, N, seed=4242, storage=h.STORE_BITS, traj_cap=generations, stream=stream)
    p.init_population()
    p.fitness()
    cands = shape_candidates(m)
    ms = {c: 0.0 for c in cands}
    for _ in range(2):             # alternate the candidates so that drift of the population evens out
        for c in cands:
            h.set_fused_shape(p, *c)
            h.step_multi([p], 4)   # warm-up
            ms[c] += _time([p], generations, stream)
    p.close()
    best = min(ms, key=ms.get)
    res = {"tpp": best[0], "nch": best[1],
           "ms_per_generation": {f"tpp{c[0]}_nch{c[1]}": v / (2 * generations) for c, v in ms.items()}}
    if use_cache:
        cache = _load()
        cache[key] = res
        _save(cache)
    return res


def tune_fused(specs, generations: int = 32, stream=None, use_cache: bool = True) -> dict:
    """specs: list of (m, N).  Tuned shape per population and the block count
    of the joint launch: {"shapes": [(tpp, nch)], "blocks": b, ...}."""
    shapes = [tune_shape(m, N, generations, stream, use_cache) for m, N in specs]
    sh = [(s["tpp"], s["nch"]) for s in shapes]
    key = _key(specs) + "|" + ",".join(f"t{a}n{b}" for a, b in sh)
    cache = _load() if use_cache else {}
    if key in cache:
        return cache[key]
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    candidates = sorted({max(1, sms // 4), sms // 2, (3 * sms) // 4, sms})
    stream = stream if stream is not None else torch.cuda.Stream()
    pops = []
    for idx, (m, N) in enumerate(specs):
        p = h.Population(m, N, seed=12345, pop_id=idx, storage=h.STORE_BITS, traj_cap=generations, stream=stream)
        h.set_fused_shape(p, *sh[idx])
        p.init_population()
        p.fitness()
        pops.append(p)
    times = {}
    for b in candidates:
        h.set_fused_grid(pops[0], b)
        h.step_multi(pops, 4)  # warm-up
        times[b] = _time(pops, generations, stream)
    for p in pops:
        p.close()
    best = min(times, key=times.get)
    res = {"blocks": int(best), "shapes": [list(x) for x in sh],
           "ms_per_generation": {str(k): v / generations for k, v in times.items()}}
    if use_cache:
        cache = _load()
        cache[key] = res
        _save(cache)
    return res


def apply_fused(pops, tuned: dict):
    """Sets the tuned shapes and block count on the populations of a launch."""
    for p, (tpp, nch) in zip(pops, tuned["shapes"]):
        h.set_fused_shape(p, tpp, nch)
    h.set_fused_grid(pops[0], tuned["blocks"])


def tune_fused_grid(specs, generations: int = 32, stream=None, use_cache: bool = True) -> int:
    """The block count alone (default shapes): kept for callers that tune nothing else."""
    key = _key(specs)
    cache = _load() if use_cache else {}
    if key in cache and "blocks" in cache[key]:
        return int(cache[key]["blocks"])
    res = tune_fused(specs, generations, stream, use_cache)
    return int(res["blocks"])


GRAM_PATHS = (h.PATH_INT32, h.PATH_IMMA, h.PATH_POPC, h.PATH_FP8, h.PATH_BF16, h.PATH_FP8_WARP)


def tune_gram_path(storage: int, m: int, kind: int, gib: float = 2.0, reps: int = 3, use_cache: bool = True,
                   apply: bool = True) -> dict:
    """Fastest exact Gram path for (storage, m, kind) on this GPU; applied as
    the process-wide GA_PATH_AUTO choice unless apply is False."""
    key = f"{_gpu()}|path|s{storage}m{m}k{kind}"
    cache = _load() if use_cache else {}
    if key not in cache:
        P = max(1024, int(gib * (1 << 30)) // (m * m))
        pop = h.empty_population(storage, m, P)
        h.ga_init_batch(pop, storage, m, P, 31)
        fit = torch.zeros(P, dtype=torch.int32, device="cuda")
        ref = None
        ms = {}
        for path in GRAM_PATHS:
            try:
                h.ga_fitness_batch(pop, storage, m, P, kind, path, fit)
            except h.GAError:
                continue          # the path does not compute this fitness of this storage
            torch.cuda.synchronize()
            if ref is None:
                ref = fit.clone()
            elif not torch.equal(ref, fit):
                raise RuntimeError(f"Gram path {path} disagrees with path {GRAM_PATHS[0]} at m={m}")
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                h.ga_fitness_batch(pop, storage, m, P, kind, path, fit)
            e1.record()
            e1.synchronize()
            ms[path] = e0.elapsed_time(e1) / reps
        del pop, fit
        best = min(ms, key=ms.get)
        cache_entry = {"path": int(best), "P": P, "ms": {str(k): v for k, v in ms.items()}}
        if use_cache:
            cache = _load()
            cache[key] = cache_entry
            _save(cache)
        cache = {key: cache_entry}
    res = cache[key]
    if apply:
        h.set_auto_path(storage, m, kind, int(res["path"]))
    return res
