"""Throughput of the GA population step on GB300 (one JSON line on stdout).

Workload: m = 20, P = 40,000 balanced +-1 matrices (N = 10,000; the paper's
stated scale), fitness = sum over i < j of G_ij^2, one balanced pair-flip per
child (NC = NR = 1), Philox seed 1, bit storage.  A step is the whole
1,000-generation run of that workload (STEP_GENS generations of the whole hot
path: selection, survivor placement, crossover, mutation, offspring fitness,
best individual), run by the fused persistent generation kernel through the
C ABI (ga_step).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

value     generations/s of the fused path, inputs resident in HBM, CUDA events
          on the context's stream; the L2 cache is flushed (256 MiB write)
          before every step, outside the timed events.
e2e       the same metric with the population and fitness copied in from
          pinned host memory, and the final population, fitness and the
          step's best-fitness trajectory copied back, every step, inside the
          timed region (wall clock).
plain     the one-kernel-per-operator path on the same workload.
roofline  the persistent kernel's algorithmic bytes (P*S + 16P per
          generation) against the measured HBM copy bandwidth.
m32plus   orders m >= 32: the m = 100 GA with full and incremental fitness
          and the batched Gram + F_sq at m = 32..256 (8 GiB of int8 each),
          with roofline fractions against their algorithmic work and sampled
          checks against the oracle (bounded: about a minute).
cpu_baseline  the CPU oracle on a bounded sample of the same workload.
--impl reference times the oracle alone (the reference arm of this build).
Under torchrun each rank runs an independent replica population
(pop_id = rank); value sums the generations of all ranks over the slowest
rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

M, N, SEED, NC, NR = 20, 10_000, 1, 1, 1
P = 4 * N
STEP_GENS = 1000
# the same metric and workload on both arms (the reference arm's steps are shorter)
METRIC = "GA generations/s at m=20, P=40k"
WORKLOAD = "m=20, P=40,000, F_sq, NC=NR=1, seed 1"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# DRAM read + write bytes of one k_fused launch of this workload (ncu,
# dram__bytes_read.sum + dram__bytes_write.sum, caches flushed before the
# launch), with the SHA-256 of the kernel sources the capture was taken on:
# when the sources differ the number no longer describes the kernel that
# runs and the bench line reports traffic as null.
FUSED_M20_TRAFFIC = {"bytes": 8406016.0, "generations_per_launch": 64,
                     "sources_sha256": "5223cf4c6266eb7b4f6d22968e58cb45aa568c99b45c05aa96b9ed33f96bc4c7"}
FUSED_SOURCES = ("k_fused.cu", "common.cuh", "inc_plan.cuh", "kernels.cuh")


def fused_sources_sha256():
    """SHA-256 over the sources the persistent generation kernel is built from."""
    import hashlib
    hsh = hashlib.sha256()
    for f in FUSED_SOURCES:
        with open(os.path.join(ROOT, "paper_2208_14961_gb300", "csrc", f), "rb") as fh:
            hsh.update(fh.read())
    return hsh.hexdigest()


def job_rate(local_time, units_per_rank, world, reduce_max=None, device=None):
    """Whole-job throughput of `world` replica ranks: every rank processed
    `units_per_rank` units in `local_time` (any time unit); the job takes as
    long as its slowest rank, so the rate is world * units / max over ranks
    of the time.  `reduce_max` is a collective MAX over ranks (None on one
    rank).  Returns (rate per time unit, max time)."""
    import torch
    t = torch.tensor([float(local_time)], dtype=torch.float64, device=device)
    if world > 1 and reduce_max is not None:
        reduce_max(t)
    slowest = float(t.item())
    return world * units_per_rank / slowest, slowest


def bytes_per_generation(m=M, N=N):
    """Algorithmic HBM bytes of one generation of the method (bit storage):
    read the 2N parents and write the 2N offspring, P*S bytes, plus 16 bytes
    per individual of fitness, keys and indices."""
    w = (m + 31) // 32
    return 4 * N * m * w * 4 + 16 * 4 * N


def impl_bytes_per_generation(m=M, N=N):
    """Bytes this implementation moves per generation (context, not the
    roofline's numerator): it also places the 2N parents physically in the
    next population buffer, i.e. read 2N parents, write all 4N slots, read
    and write the 4N fitness words, read the survivor-order row (2N words)."""
    w = (m + 31) // 32
    mat = m * w * 4
    return 2 * N * mat + 4 * N * mat + 2 * 4 * N * 4 + 2 * N * 4


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.proc, self.lines = index, None, []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_sample(seconds=12.0, min_gens=3, threads=None):
    """Times the CPU oracle on the same workload for a bounded number of
    generations (about `seconds` of host CPU time), on all host cores or on
    `threads` of them."""
    import oracle
    if threads:
        prev = oracle.num_threads()
        oracle.set_num_threads(threads)
        try:
            return oracle_sample(seconds, min_gens)
        finally:
            oracle.set_num_threads(prev)
    pop = oracle.init_population(M, P, SEED)
    F = oracle.fitness(pop, oracle.FIT_SQ)
    t0 = time.perf_counter()
    gens = 0
    while gens < min_gens or time.perf_counter() - t0 < seconds:
        oracle.run(pop, F, N, NC, NR, oracle.FIT_SQ, SEED, 0, gens, 1)
        gens += 1
        if gens >= 2000:
            break
    dt = time.perf_counter() - t0
    return gens / dt, gens, dt, oracle.num_threads()


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle as it stands, on the host cores."""
    if rank != 0:
        return
    import oracle
    pop = oracle.init_population(M, P, SEED)
    F = oracle.fitness(pop, oracle.FIT_SQ)
    sample = 4  # generations per step: a bounded sample of a 50-generation step
    g = 0
    for _ in range(args.warmup):
        oracle.run(pop, F, N, NC, NR, oracle.FIT_SQ, SEED, 0, g, sample)
        g += sample
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.run(pop, F, N, NC, NR, oracle.FIT_SQ, SEED, 0, g, sample)
        g += sample
    dt = time.perf_counter() - t0
    gps = args.steps * sample / dt
    line = {
        "impl": "reference",
        "metric": METRIC, "arm": "CPU oracle (int8 matrices)",
        "value": gps, "unit": "generations/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "generations_per_step": sample, "global_batch": P},
        "cpu_baseline": {"value": gps, "unit": "generations/s", "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"{sample} generations per step, {args.steps} steps"},
        "e2e": {"value": gps, "unit": "generations/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


GRAM_PATHS = [  # name, storage, path
    ("int32", 0, 1), ("imma", 0, 2), ("popc_int8", 0, 5), ("popc_bits", 1, 5), ("fp8", 2, 3), ("bf16", 3, 4),
    ("fp8_warp", 2, 6),
]


def popc_per_dot(m):
    """Population counts per column pair of the popcount Gram: W = ceil(m/32)
    XOR words, reduced by carry-save adders for W >= 3 (2 counts at W = 3,
    3 at W = 4..7, 4 at W = 8)."""
    W = (m + 31) // 32
    return W if W <= 2 else 2 if W == 3 else 3 if W <= 7 else 4


def _library_gemm_tflops(kind, n=8192, reps=20):
    """Dense n x n x n GEMM rate of the vendor library (cuBLAS / cuBLASLt via
    torch) in TFLOP/s: "bf16" (torch.mm) or "fp8" (e4m3 x e4m3 -> bf16,
    torch._scaled_mm); None where the installed torch lacks the call."""
    import torch
    try:
        a = torch.randn(n, n, device="cuda")
        b = torch.randn(n, n, device="cuda")
        if kind == "bf16":
            a, b = a.to(torch.bfloat16), b.to(torch.bfloat16)
            run = lambda: torch.mm(a, b)
        else:
            a8, b8 = a.to(torch.float8_e4m3fn), b.to(torch.float8_e4m3fn)
            one = torch.ones((), device="cuda", dtype=torch.float32)
            bt = b8.t()  # column-major second operand
            run = lambda: torch._scaled_mm(a8, bt, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)
        for _ in range(3):
            run()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        for _ in range(reps):
            run()
        ev[1].record()
        ev[1].synchronize()
        return 2.0 * n ** 3 * reps / (ev[0].elapsed_time(ev[1]) / 1e3) / 1e12
    except Exception:
        return None


def peaks_report(args):
    """The microbenchmark rates the roofline fractions use, plus SM count,
    L2 size and the library's dense bf16 / fp8 GEMM rates (one JSON line)."""
    import torch

    from paper_2208_14961_gb300 import peaks
    prop = torch.cuda.get_device_properties(0)
    r = {k: peaks.rate(k) for k in peaks.KINDS}
    line = {"gpu": prop.name, "sms": prop.multi_processor_count,
            "l2_bytes": getattr(prop, "L2_cache_size", None),
            "popc_per_s": r["popc_chain"], "dp4a_per_s": r["dp4a"], "imad_per_s": r["imad"],
            "mma_sync_s8_mac_per_s": r["imma_s8"], "mma_sync_e4m3_mac_per_s": r["mma_e4m3"],
            "l2_read_bytes_per_s": r["l2_read_bytes"], "dfma_per_s": r["dfma"], "ffma_per_s": r["ffma"],
            "grid_barrier_us": (1e6 / r["grid_barriers"]) if r["grid_barriers"] > 0 else None,
            "library_gemm_tflops": {"bf16": _library_gemm_tflops("bf16"), "fp8_e4m3": _library_gemm_tflops("fp8")},
            "hbm_gbs": _peaks()[0], "hbm_source": _peaks()[1]}
    print(json.dumps(line), flush=True)


def gram_sweep(args):
    """Precision sweep of the batched Gram + F_sq alone: balanced +-1
    populations of `--gram-gb` GiB of int8 (seed 2) at each order, every
    path on its own storage format; one JSON line per (m, path) with the
    time per pass, matrices/s, achieved GB/s of its storage, the bound
    roof and an exactness check of 256 sampled slots against the oracle."""
    import numpy as np
    import torch

    import oracle
    from paper_2208_14961_gb300.build import build
    build()
    from paper_2208_14961_gb300 import hadga as h
    from paper_2208_14961_gb300 import peaks

    hbm, hbm_kind = _peaks()
    rates = {k: peaks.rate(k) for k in ("popc_chain", "dp4a", "mma_e4m3")}
    print(json.dumps({"peaks": {"hbm_gbs": hbm, "hbm_source": hbm_kind, "popc_per_s": rates["popc_chain"],
                                "dp4a_per_s": rates["dp4a"], "mma_sync_e4m3_mac_per_s": rates["mma_e4m3"]}}),
          flush=True)
    rng = np.random.default_rng(7)
    for m in [int(x) for x in args.gram_ms.split(",")]:
        P = int(args.gram_gb * (1 << 30)) // (m * m)
        D = m * (m - 1) // 2
        W = (m + 31) // 32
        for name, storage, path in GRAM_PATHS:
            if args.gram_paths and name not in args.gram_paths.split(","):
                continue
            try:
                pop = h.empty_population(storage, m, P)
            except RuntimeError as e:
                print(json.dumps({"m": m, "path": name, "skipped": f"allocation: {e}"[:200]}), flush=True)
                continue
            fit = torch.zeros(P, dtype=torch.int32, device="cuda")
            h.ga_init_batch(pop, storage, m, P, 2)
            try:
                h.ga_fitness_batch(pop, storage, m, P, h.FIT_SQ, path, fit)
            except h.GAError as e:
                print(json.dumps({"m": m, "path": name, "skipped": str(e)[:200]}), flush=True)
                del pop, fit
                torch.cuda.empty_cache()
                continue
            torch.cuda.synchronize()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            reps = 5
            ev[0].record()
            for _ in range(reps):
                h.ga_fitness_batch(pop, storage, m, P, h.FIT_SQ, path, fit)
            ev[1].record()
            ev[1].synchronize()
            sec = ev[0].elapsed_time(ev[1]) / 1e3 / reps
            # exactness on sampled slots
            idx_np = np.sort(rng.choice(P, size=min(256, P), replace=False))
            idx = torch.as_tensor(idx_np, device="cuda")
            ref = oracle.fitness(oracle.init_slots(m, idx_np, 2), oracle.FIT_SQ)
            got = fit.index_select(0, idx).cpu().numpy().view(np.uint32).astype(np.uint64)
            exact = bool(np.array_equal(ref, got))
            nbytes = P * h.storage_bytes(storage, m)
            t_mem = nbytes / (hbm * 1e9)
            if name == "popc_bits" or name == "popc_int8":
                ops, peak, unit = P * D * popc_per_dot(m), rates["popc_chain"], "popc"
            elif name == "int32":
                ops, peak, unit = P * D * (m // 4), rates["dp4a"], "dp4a"
            elif name in ("imma", "fp8_warp") and m % 32 == 0:
                mt, ct, ks = m // 16, m // 8, m // 32
                tiles = sum(ct - 2 * ri for ri in range(mt))
                ops, peak, unit = P * tiles * ks * 4096, rates["mma_e4m3"], "e4m3 MAC"
            else:
                ops, peak, unit = None, None, None
            t_cmp = ops / peak if ops else 0.0
            bound = "hbm" if t_mem >= t_cmp else "alu" if name not in ("imma", "fp8_warp") else "tensor"
            roof_t = max(t_mem, t_cmp)
            line = {"m": m, "path": name, "P": P, "storage_gib": nbytes / (1 << 30), "ms": sec * 1e3,
                    "matrices_per_s": P / sec, "achieved_gbs": nbytes / sec / 1e9, "bound": bound,
                    "roof_ms": roof_t * 1e3, "frac": roof_t / sec, "hbm_frac": t_mem / sec,
                    "compute_unit": unit, "compute_frac": (t_cmp / sec) if ops else None, "exact_256": exact}
            print(json.dumps(line), flush=True)
            del pop, fit
            torch.cuda.empty_cache()


# Sec. 2, Table 1: seconds per additional batched product (N = 10,000, m = 100,
# float64) on the paper's machines, from the text (CuPy on an RTX 3080: about
# 0.07 s a loop; NumPy on the host CPU: about 2.12 s a loop).
PAPER_TABLE1_CUPY_S, PAPER_TABLE1_NUMPY_S = 0.07, 2.12


def table1_workload(args):
    """The batched-Gram speed comparison of Sec. 2 (Table 1): N = 10,000
    random 100 x 100 matrices (uniform on [0, 1), seeded), each multiplied by
    its own transpose, in float64 (the paper's type) and float32.  One JSON
    line per type: seconds per batched product through ga_gram_real_batch
    with the data resident (800 MB in + 800 MB out in float64, larger than
    the L2, so no flush), end to end with the input copied in from pinned
    host memory and G copied back, the library batched product (torch.bmm)
    timed beside it, the roofline against the measured FMA rate and the HBM
    copy bandwidth, a sampled check against the oracle, and the oracle's own
    rate on a bounded sample of host cores."""
    import numpy as np
    import torch

    import oracle
    from paper_2208_14961_gb300.build import build
    build()
    from paper_2208_14961_gb300 import hadga as h
    from paper_2208_14961_gb300 import peaks

    Nm, m = args.t1_n, args.t1_m
    hbm, hbm_kind = _peaks()
    gen = torch.Generator(device="cuda")
    for dtype, name, fma_kind in ((torch.float64, "f64", "dfma"), (torch.float32, "f32", "ffma")):
        fma_rate = peaks.rate(fma_kind)
        gen.manual_seed(11)
        q = torch.rand((Nm, m, m), dtype=dtype, device="cuda", generator=gen)
        g = torch.empty_like(q)
        reps = args.t1_reps
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        launches0 = h.kernel_launches()
        for _ in range(3):
            h.ga_gram_real_batch(q, g)
        torch.cuda.synchronize()
        ev[0].record()
        for _ in range(reps):
            h.ga_gram_real_batch(q, g)
        ev[1].record()
        ev[1].synchronize()
        sec = ev[0].elapsed_time(ev[1]) / 1e3 / reps
        launches = h.kernel_launches() - launches0
        # the library product of the paper's listing: matmul(Q^T, Q), all m^2 entries
        qt = q.transpose(1, 2)
        for _ in range(2):
            torch.bmm(qt, q)
        torch.cuda.synchronize()
        ev[0].record()
        for _ in range(reps):
            torch.bmm(qt, q)
        ev[1].record()
        ev[1].synchronize()
        sec_lib = ev[0].elapsed_time(ev[1]) / 1e3 / reps
        # end to end: pinned host input in, G out, every product
        qh = q.cpu().pin_memory()
        gh = torch.empty_like(qh).pin_memory()
        s = torch.cuda.current_stream()
        t0 = time.perf_counter()
        e2e_reps = max(1, reps // 4)
        for _ in range(e2e_reps):
            q.copy_(qh, non_blocking=True)
            h.ga_gram_real_batch(q, g, stream=s)
            gh.copy_(g, non_blocking=True)
        torch.cuda.synchronize()
        sec_e2e = (time.perf_counter() - t0) / e2e_reps
        # sampled check against the oracle (the summation bound of both sides)
        idx = np.random.default_rng(12).choice(Nm, 32, replace=False)
        tidx = torch.as_tensor(idx, device="cuda")
        Qs = q[tidx].cpu().numpy().astype(np.float64)
        Gs = g[tidx].cpu().numpy().astype(np.float64)
        u = 2.0 ** -53 if dtype == torch.float64 else 2.0 ** -24
        gam = lambda n, uu: n * uu / (1 - n * uu)
        tol = 1.001 * (gam(m, u) + gam(m, 2.0 ** -53)) * oracle.gram_real(np.abs(Qs))
        ok = bool(np.all(np.abs(Gs - oracle.gram_real(Qs)) <= tol))
        # oracle on a bounded sample of host cores
        ns = max(1, min(Nm, args.t1_oracle_matrices))
        Qc = Qs if ns <= len(Qs) else q[:ns].cpu().numpy().astype(np.float64)
        Qc = Qc[:ns]
        t0 = time.perf_counter()
        oracle.gram_real(Qc)
        t_orc = (time.perf_counter() - t0) * Nm / ns
        elem = q.element_size()
        fma_alg = m * m * (m + 1) // 2          # one FMA per term of each distinct entry
        bytes_alg = 2 * m * m * elem            # read Q, write G
        t_fma = Nm * fma_alg / fma_rate
        t_mem = Nm * bytes_alg / (hbm * 1e9)
        bound = "fma" if t_fma >= t_mem else "hbm"
        line = {"metric": "batched Gram seconds per product (Table 1)", "dtype": name, "N": Nm, "m": m,
                "value": sec, "unit": "s", "higher_is_better": False, "matrices_per_s": Nm / sec,
                "gpu_launches": launches // (reps + 3),
                "e2e": {"value": sec_e2e, "unit": "s", "h2d_bytes_per_step": Nm * m * m * elem,
                        "d2h_bytes_per_step": Nm * m * m * elem},
                "library_bmm_s": sec_lib,
                "roofline": {"bound": bound, "fma_per_s_achieved": Nm * fma_alg / sec,
                             "fma_per_s_peak": fma_rate, "fma_frac": t_fma / sec,
                             "gbs_achieved": Nm * bytes_alg / sec / 1e9, "gbs_peak": hbm, "hbm_frac": t_mem / sec,
                             "peak_source": f"FMA rate measured by the peaks microbenchmark; HBM {hbm_kind}"},
                "paper_s_per_loop": {"cupy_rtx3080": PAPER_TABLE1_CUPY_S, "numpy_cpu": PAPER_TABLE1_NUMPY_S},
                "cpu_baseline": {"value": t_orc, "unit": "s", "cores": oracle.num_threads(), "kind": "oracle",
                                 "sample": f"{ns} matrices, scaled to N={Nm}"},
                "within_bound_32_sampled": ok}
        print(json.dumps(line), flush=True)
        del q, g, qh, gh
        torch.cuda.empty_cache()


MIXED_ORDERS = (12, 16, 20, 24, 28, 32, 36)


def _mixed_rate(h, specs, stream, gens, tuned):
    """Generations/s of the mixed-order launch as CUDA-graph replays of
    50-generation chunks, with the tuned shapes or (tuned None) the
    defaults (four threads per pair, the cost model's chunking, one block
    per SM)."""
    import torch

    from paper_2208_14961_gb300 import autotune
    pops = []
    for i, (m, N) in enumerate(specs):
        p = h.Population(m, N, seed=3, pop_id=i, fitness=h.FIT_SQ, storage=h.STORE_BITS, traj_cap=512,
                         stream=stream)
        p.init_population()
        p.fitness()
        pops.append(p)
    if tuned:
        autotune.apply_fused(pops, tuned)
    h.step_multi_graph(pops, 50, 50)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    h.step_multi_graph(pops, gens, 50)
    e1.record(stream)
    e1.synchronize()
    for p in pops:
        p.close()
    return gens / (e0.elapsed_time(e1) / 1e3)


def mixed_workload(args):
    """Batched mixed orders in one persistent launch: one population per
    order m in {12, ..., 36}, P = 4(500 + U[0, 4500]) each (Philox stream
    CONFIG, seed 3; pop_id = order position), F_sq, NC = NR = 1, 500
    generations as CUDA-graph replays of 50-generation chunks, block count
    from the autotuner.  Prints one JSON line."""
    import torch

    import oracle
    from paper_2208_14961_gb300.build import build
    build()
    from paper_2208_14961_gb300 import autotune
    from paper_2208_14961_gb300 import hadga as h

    specs = [(m, oracle.mixed_N(3, i)) for i, m in enumerate(MIXED_ORDERS)]
    stream = torch.cuda.Stream()
    tuned = autotune.tune_fused(specs, stream=stream)
    default_gps = None
    if args.mixed_compare_default:
        default_gps = _mixed_rate(h, specs, stream, args.mixed_gens, None)

    def fresh():
        pops = []
        for i, (m, N) in enumerate(specs):
            p = h.Population(m, N, seed=3, pop_id=i, fitness=h.FIT_SQ, storage=h.STORE_BITS, traj_cap=512,
                             stream=stream)
            p.init_population()
            p.fitness()
            pops.append(p)
        autotune.apply_fused(pops, tuned)
        return pops

    gens, chunk = args.mixed_gens, 50
    pops = fresh()
    h.step_multi_graph(pops, chunk, chunk)  # warm-up (also builds the graph path once)
    torch.cuda.synchronize()
    pops = fresh()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    h.step_multi_graph(pops, gens, chunk)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    total_P = sum(4 * N for _, N in specs)
    exact = None
    if args.mixed_check:
        exact = True
        for i, ((m, N), p) in enumerate(zip(specs, pops)):
            ref = oracle.init_population(m, 4 * N, 3, i)
            F = oracle.fitness(ref, oracle.FIT_SQ)
            oracle.run(ref, F, N, 1, 1, oracle.FIT_SQ, 3, i, 0, gens)
            exact = exact and bool((p.as_int8() == ref).all()) and bool((p.fitness_host() == F).all())
    line = {"workload": "mixed orders 12..36 in one persistent launch", "orders": list(MIXED_ORDERS),
            "P": [4 * N for _, N in specs], "generations": gens, "graph_chunk": chunk,
            "autotuned_blocks": tuned["blocks"],
            "autotuned_shapes": {str(m): {"threads_per_pair" if m <= 32 else "warp_gram_chunks":
                                          (t if m <= 32 else n)} for (m, _), (t, n) in zip(specs, tuned["shapes"])},
            "ms": ms, "generations_per_s": gens / (ms / 1e3),
            "evals_per_s": gens * (total_P // 2) / (ms / 1e3), "exact_vs_oracle": exact,
            "default_shapes_generations_per_s": default_gps}
    for p in pops:
        p.close()
    print(json.dumps(line), flush=True)


# Sec. 4.2, Table 2 of the paper: seconds for 10^4 generations at P = 40,000,
# NC = 4, NR = 2 on an RTX 3080 (CuPy, int8 matmul), fitness F1 and F2.
PAPER_TABLE_SECONDS = {20: (60.50, 59.38), 40: (103.15, 99.84), 60: (176.28, 170.20),
                       80: (275.92, 256.59), 100: (416.68, 381.38)}


def _popc_roof(gens_per_s, m, offspring):
    """The generation rate against the population-count roof of its Gram
    work: every offspring's m(m-1)/2 column pairs at popc_per_dot(m) counts
    each, over the measured count rate of the peak microbenchmark."""
    from paper_2208_14961_gb300 import peaks
    peak = peaks.rate("popc_chain")
    achieved = gens_per_s * offspring * (m * (m - 1) // 2) * popc_per_dot(m)
    return {"bound": "alu", "unit": "popc/s", "achieved": achieved, "peak": peak, "frac": achieved / peak,
            "work": "offspring Gram popcounts per generation", "peak_source": "measured (peaks microbenchmark)"}


def table3_workload(args):
    """The paper's fitness-comparison workload (Sec. 4.2): m in {20, 40, 60,
    80, 100}, P = 40,000 balanced +-1 matrices (seed 5), NC = 4 columns and
    NR = 2 row pairs per mutation, fitness F1 and F2.  Each (m, fitness) runs
    `--t3-gens` generations of the fused path (bit storage) in ga_step calls
    of 50 after a warm-up call; the first 50 generations are also run by the
    one-kernel-per-operator path and must give the same population and
    fitness.  One JSON line per (m, fitness) with generations/s, evaluations/s
    in the paper's convention (all P per generation) and the paper's RTX 3080
    rate for the same m and fitness (context: other hardware)."""
    import numpy as np
    import torch

    from paper_2208_14961_gb300.build import build
    build()
    from paper_2208_14961_gb300 import hadga as h

    N, seed, chunk = 10_000, 5, 50
    gens = max(chunk, args.t3_gens // chunk * chunk)
    stream = torch.cuda.Stream()
    for m in [int(x) for x in args.t3_ms.split(",")]:
        for kind, kname in ((h.FIT_ABS, "F1"), (h.FIT_NNZ, "F2")):
            def fresh():
                p = h.Population(m, N, seed=seed, NC=4, NR=2, fitness=kind, storage=h.STORE_BITS,
                                 traj_cap=chunk, stream=stream)
                p.init_population()
                p.fitness()
                return p
            a, b = fresh(), fresh()
            a.step(chunk)
            b.step_plain(chunk)
            a.sync()
            b.sync()
            exact = bool(np.array_equal(a.as_int8(), b.as_int8())) and bool(
                np.array_equal(a.fitness_host(), b.fitness_host()))
            b.close()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(gens // chunk):
                a.step(chunk)
            e1.record(stream)
            e1.synchronize()
            sec = e0.elapsed_time(e1) / 1e3
            best = a.best()
            a.close()
            gps = gens / sec
            paper_s = PAPER_TABLE_SECONDS.get(m, (None, None))[0 if kind == h.FIT_ABS else 1]
            paper_gps = 1e4 / paper_s if paper_s else None
            line = {"workload": "paper Sec. 4.2 fitness comparison", "m": m, "P": 4 * N, "NC": 4, "NR": 2,
                    "fitness": kname, "generations": gens, "ms": sec * 1e3, "generations_per_s": gps,
                    "evals_per_s_paper_convention": gps * 4 * N, "fused_equals_plain_50": exact,
                    "best_fitness": int(best[1]),
                    "paper_rtx3080_generations_per_s": paper_gps,
                    "over_paper": (gps / paper_gps) if paper_gps else None,
                    "roofline": _popc_roof(gps, m, 2 * N)}
            print(json.dumps(line), flush=True)


# Sec. 4.4 of the paper: runs that found Hadamard matrices with fitness F2 on
# an RTX 3080: (m, N, NC, NR, generations, seconds).
PAPER_SEARCHES = [(20, 1000, 2, 8, 258_875, 517), (24, 1000, 2, 10, 9_576_814, 19_997),
                  (28, 10_000, 1, 10, 428_082, 3_054), (32, 20_000, 1, 12, 7_472_853, 94_923)]


def search_workload(args):
    """Time to a Hadamard matrix (Sec. 4.4): for each order of the paper's
    successful searches, with its population size, mutation parameters and
    fitness F2, run the fused path in ga_step calls of `--search-chunk`
    generations with stop_at_zero until the best fitness is 0 or
    `--search-seconds` pass; several seeds (`--search-seeds`).  A matrix found
    is read back and checked on the host: Q^T Q = m I.  One JSON line per run
    with the generations and seconds taken, next to the paper's run (one run
    of a stochastic search on other hardware: context, not a target)."""
    import numpy as np

    from paper_2208_14961_gb300.build import build
    build()
    from paper_2208_14961_gb300 import hadga as h

    orders = [int(x) for x in args.search_ms.split(",")]
    for (m, N, NC, NR, p_gens, p_sec) in PAPER_SEARCHES:
        if m not in orders:
            continue
        for seed in range(args.search_seeds):
            pop = h.Population(m, N, seed=100 + seed, NC=NC, NR=NR, fitness=h.FIT_NNZ, storage=h.STORE_BITS,
                               traj_cap=args.search_chunk)
            pop.set_strict(True)   # the persistent kernel, never the plain fallback
            pop.init_population()
            pop.fitness()
            pop.sync()
            gens, found = 0, False
            t0 = time.perf_counter()
            while time.perf_counter() - t0 < args.search_seconds:
                done = pop.step(args.search_chunk, stop_at_zero=True)
                gens += done
                if done < args.search_chunk:
                    found = True
                    break
            pop.sync()
            sec = time.perf_counter() - t0
            line = {"workload": "paper Sec. 4.4 search", "m": m, "P": 4 * N, "NC": NC, "NR": NR, "fitness": "F2",
                    "seed": 100 + seed, "found": found, "generations": gens, "seconds": sec,
                    "generations_per_s": gens / sec if sec > 0 else None,
                    "paper_rtx3080": {"generations": p_gens, "seconds": p_sec}}
            slot, best = pop.best()
            line["best_fitness"] = int(best)
            if found:
                Q = pop.get_slot(slot).astype(np.int64)
                line["verified_QtQ_eq_mI"] = bool(np.array_equal(Q.T @ Q, m * np.eye(m, dtype=np.int64)))
            pop.close()
            print(json.dumps(line), flush=True)


# Sec. 4.3, Tables 4 and 5 of the paper (the tables numbered 3 and 4 in its
# source): mean generations to a Hadamard matrix of order 12 and 16, F2,
# 10 runs per cell, rows NR = 1..4, columns NC = 1..4 (the order-16 cells
# NR = 1, NC = 2..4 are those where most runs found none).
PAPER_TABLE4_M12 = [[34.2, 35.8, 37.4, 35.8], [32.3, 38.8, 40.5, 43.4], [35.2, 42.6, 47.5, 50.7],
                    [36.3, 46.0, 49.9, 65.7]]
PAPER_TABLE5_M16 = [[130.1, 119.4, 116.0, 115.5], [121.0, 181.3, 135.0, 168.7], [120.0, 158.1, 165.9, 202.7],
                    [120.2, 166.2, 236.2, 301.6]]


def table45_workload(args):
    """The convergence statistics of Sec. 4.3 (Tables 4 and 5): for m = 12
    and 16, F2, N = 1000 (the listing's default population, P = 4,000), every
    NC, NR in 1..4, `--t45-seeds` seeded runs of the fused path with
    stop_at_zero, capped at `--t45-cap` generations.  One JSON line per
    (m, NC, NR): runs that found a Hadamard matrix (each checked Q^T Q = m I
    on the host), the mean and median generations of those runs, and the
    paper's mean for the cell (a plausibility band: the paper's random
    streams and its int64/int32 index reading differ from this build's)."""
    import numpy as np

    from paper_2208_14961_gb300.build import build
    build()
    from paper_2208_14961_gb300 import hadga as h

    tables = {12: PAPER_TABLE4_M12, 16: PAPER_TABLE5_M16}
    for m in [int(x) for x in args.t45_ms.split(",")]:
        for NR in range(1, 5):
            for NC in range(1, 5):
                gens_found, verified = [], True
                t0 = time.perf_counter()
                for seed in range(args.t45_seeds):
                    pop = h.Population(m, 1000, seed=1000 + seed, NC=NC, NR=NR, fitness=h.FIT_NNZ,
                                       storage=h.STORE_BITS, traj_cap=args.t45_cap)
                    pop.set_strict(True)
                    pop.init_population()
                    pop.fitness()
                    done = pop.step(args.t45_cap, stop_at_zero=True)
                    slot, best = pop.best()
                    if best == 0:
                        Q = pop.get_slot(slot).astype(np.int64)
                        verified = verified and bool(np.array_equal(Q.T @ Q, m * np.eye(m, dtype=np.int64)))
                        gens_found.append(done)
                    pop.close()
                line = {"workload": "paper Sec. 4.3 convergence (Tables 4-5)", "m": m, "NC": NC, "NR": NR,
                        "fitness": "F2", "P": 4000, "runs": args.t45_seeds, "cap": args.t45_cap,
                        "found": len(gens_found), "verified_QtQ_eq_mI": verified,
                        "mean_generations_found": float(np.mean(gens_found)) if gens_found else None,
                        "median_generations_found": float(np.median(gens_found)) if gens_found else None,
                        "paper_mean_generations": tables[m][NR - 1][NC - 1] if m in tables else None,
                        "seconds": time.perf_counter() - t0}
                print(json.dumps(line), flush=True)


def incremental_workload(args):
    """Incremental Gram-delta fitness (a7) on m=100, P=20,000 bit-packed
    balanced matrices (seed 4, F_sq, NC = NR = 1) for `--inc-gens`
    generations (default 10,000) in ga_step calls of 100 generations.  After
    every call a full recomputation of every slot's Gram and fitness on the
    GPU is compared with the incrementally kept values; the population after
    the first 100 generations is compared with the oracle's; the same run
    with full recomputation gives the comparison rate and must produce the
    same best-fitness trajectory.  Prints one JSON line."""
    import numpy as np
    import torch

    import oracle
    from paper_2208_14961_gb300.build import build
    build()
    from paper_2208_14961_gb300 import hadga as h

    m, N, seed, every = 100, 5000, 4, 100
    gens = max(every, args.inc_gens // every * every)
    stream = torch.cuda.Stream()

    def fresh(inc):
        p = h.Population(m, N, seed=seed, fitness=h.FIT_SQ, storage=h.STORE_BITS, traj_cap=gens, stream=stream)
        p.init_population()
        p.fitness()
        if inc:
            p.set_incremental(True)
        p.sync()
        return p

    w = fresh(True)
    w.step(every)
    w.sync()
    w.close()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out, trajs, snap = {}, {}, None
    checks, mismatches = 0, 0
    for mode in ("incremental", "full"):
        p = fresh(mode == "incremental")
        ms = 0.0
        for c in range(gens // every):
            e0.record(stream)
            p.step(every)
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
            if mode == "incremental":
                ent, fit = p.check_incremental()
                checks += 1
                mismatches += ent + fit
                if c == 0:
                    snap = (p.as_int8(), p.fitness_host())
        trajs[mode] = p.trajectory()[0].astype(np.uint64)
        out[mode] = {"ms": ms, "generations_per_s": gens / (ms / 1e3),
                     "evals_per_s": gens * 2 * N / (ms / 1e3)}
        p.close()
    ref = oracle.init_population(m, 4 * N, seed, 0)
    F = oracle.fitness(ref, oracle.FIT_SQ)
    oracle.run(ref, F, N, 1, 1, oracle.FIT_SQ, seed, 0, 0, every)
    exact_prefix = bool((snap[0] == ref).all()) and bool((snap[1] == F).all())
    t = trajs["incremental"]
    marks = [g for g in (1, 10, 100, 1000, 10000, gens) if g <= len(t)]
    line = {"workload": "m=100, P=20,000, bit storage, F_sq, NC=NR=1, seed 4, incremental Gram-delta fitness",
            "generations": gens, "check_every": every,
            "incremental": out["incremental"], "full_recompute": out["full"],
            "incremental_over_full": out["full"]["ms"] / out["incremental"]["ms"],
            "full_rechecks": checks, "recheck_mismatches": mismatches,
            "oracle_prefix_generations": every, "exact_vs_oracle_prefix": exact_prefix,
            "trajectories_equal": bool(np.array_equal(trajs["incremental"], trajs["full"])),
            "best_fitness_at": {str(g): int(t[g - 1]) for g in sorted(set(marks))},
            "roofline_full": _popc_roof(out["full"]["generations_per_s"], m, 2 * N),
            "gram_bytes": 4 * N * ((m * (m - 1) // 2 + 15) // 16 * 16),
            "l2": "not flushed; population 32 MB + Gram 99 MB resident across calls"}
    print(json.dumps(line), flush=True)


PROFILE_CASES = """Named small workloads for profiling one kernel at a time (ncu -k):

  python bench.py --case <case> [--case-gens G]

fused_m20   m=20, P=40,000, bit storage: init, fitness, then G generations
            (default 8) in one persistent launch
plain_m20   the same with the one-kernel-per-operator path
inc_m100    m=100, P=20,000, bit storage, incremental Gram-delta fitness:
            init, fitness, Gram store, then G generations
full_m100   the same workload with full fitness recomputation
gram_m<M>_<path>  Gram + fitness of a population of ~1 GiB (int8 size) at
            order M with path int32 | imma | popc8 | popc | fp8 | bf16 | fp8w
real_<f32|f64>_m<M>  batched real Gram Q^T Q of 10,000 uniform random
            matrices of order M (two launches)"""


def profile_case(args):
    """Runs one named small workload (PROFILE_CASES) and prints one line."""
    import torch

    from paper_2208_14961_gb300.build import build
    build()
    from paper_2208_14961_gb300 import hadga as h
    case, gens = args.case, args.case_gens
    if case in ("fused_m20", "plain_m20"):
        p = h.Population(20, 10000, seed=1, storage=h.STORE_BITS, traj_cap=64)
        p.init_population()
        p.fitness()
        if case == "fused_m20":
            p.step(gens)
        else:
            p.step_plain(gens)
        p.sync()
        print(case, "best", p.best())
        return
    if case in ("inc_m100", "full_m100"):
        p = h.Population(100, 5000, seed=4, storage=h.STORE_BITS, traj_cap=64)
        p.init_population()
        p.fitness()
        if case == "inc_m100":
            p.set_incremental(True)
        p.step(gens)
        p.sync()
        print(case, "best", p.best())
        return
    if case.startswith("gram_m"):
        m_s, path_s = case[len("gram_m"):].split("_")
        m = int(m_s)
        paths = {"int32": (h.STORE_INT8, h.PATH_INT32), "imma": (h.STORE_INT8, h.PATH_IMMA),
                 "popc8": (h.STORE_INT8, h.PATH_POPC), "popc": (h.STORE_BITS, h.PATH_POPC),
                 "fp8": (h.STORE_E4M3, h.PATH_FP8), "bf16": (h.STORE_BF16, h.PATH_BF16),
                 "fp8w": (h.STORE_E4M3, h.PATH_FP8_WARP)}
        storage, path = paths[path_s]
        P = (1 << 30) // (m * m)
        pop = h.empty_population(storage, m, P)
        h.ga_init_batch(pop, storage, m, P, 2)
        fit = torch.zeros(P, dtype=torch.int32, device="cuda")
        for _ in range(2):
            h.ga_fitness_batch(pop, storage, m, P, h.FIT_SQ, path, fit)
        torch.cuda.synchronize()
        print(case, "P", P, "fit[0]", int(fit[0]))
        return
    if case.startswith("real_"):
        _, t, m_s = case.split("_")
        m = int(m_s[1:])
        dtype = torch.float64 if t == "f64" else torch.float32
        gen = torch.Generator(device="cuda")
        gen.manual_seed(11)
        q = torch.rand((10000, m, m), dtype=dtype, device="cuda", generator=gen)
        g = torch.empty_like(q)
        for _ in range(2):
            h.ga_gram_real_batch(q, g)
        torch.cuda.synchronize()
        print(case, "g[0,0,0]", float(g[0, 0, 0]))
        return
    raise SystemExit(f"unknown case {case}\n{PROFILE_CASES}")


# ---------------------------------------------------------------------------
# orders m >= 32 in the default line
# ---------------------------------------------------------------------------
M32_GRAM_ORDERS = (32, 64, 128, 256)
# exact Gram + F_sq paths timed per order: bit storage with popcounts, and
# GA_PATH_AUTO on e4m3 storage (warp-level FP8 MMA at m <= 64, tcgen05 at
# m = 128, 256)
M32_GRAM_PATHS = (("popc_bits", 1, 5), ("auto_e4m3", 2, 0))


def gram_algorithmic_work(m):
    """Algorithmic work of one matrix's Gram + fitness (i < j, i, j >= 1:
    D = (m-1)(m-2)/2 column dot products): D*m multiply-adds on int8 / e4m3
    storage, D*ceil(m/32) 32-bit population counts on bit storage."""
    D = (m - 1) * (m - 2) // 2
    return D * m, D * ((m + 31) // 32)


def _fp8_mac_rate():
    """Dense FP8 multiply-adds/s of this GPU, from the library's e4m3 GEMM
    (cuBLASLt through torch), else the nominal 4.5 PFLOP/s."""
    t = _library_gemm_tflops("fp8", n=8192, reps=10)
    return (t * 1e12 / 2, "library e4m3 GEMM, measured") if t else (2.25e15, "nominal 4.5 PFLOP/s dense")


def _roof_entry(achieved_time_s, t_mem, t_cmp, unit_cmp, peak_cmp, ops, nbytes, hbm):
    bound = "hbm" if t_mem >= t_cmp else unit_cmp
    roof_t = max(t_mem, t_cmp)
    return {"bound": bound, "frac": roof_t / achieved_time_s,
            "hbm": {"achieved_gbs": nbytes / achieved_time_s / 1e9, "peak_gbs": hbm, "frac": t_mem / achieved_time_s},
            "compute": {"unit": unit_cmp, "achieved_per_s": ops / achieved_time_s, "peak_per_s": peak_cmp,
                        "frac": t_cmp / achieved_time_s}}


def m32_gram_report(hbm, popc_rate, e4m3_warp_rate, fp8_rate, gib=8.0, reps=5):
    """Config 3 in the default line: per order m in {32, 64, 128, 256}, a
    balanced population of `gib` GiB of int8 (P = gib * 2^30 / m^2, seed 2),
    Gram + F_sq by each exact path of M32_GRAM_PATHS on its own storage,
    `reps` passes timed with CUDA events (inputs larger than L2), 256 sampled
    slots checked against the oracle; roofline against the path's
    algorithmic work (gram_algorithmic_work) and its storage bytes."""
    import numpy as np
    import torch

    import oracle
    from paper_2208_14961_gb300 import hadga as h
    from paper_2208_14961_gb300 import autotune
    rng = np.random.default_rng(7)
    out = []
    for m in M32_GRAM_ORDERS:
        # GA_PATH_AUTO on e4m3 storage takes the path the autotuner measured fastest here
        tuned_e4m3 = autotune.tune_gram_path(h.STORE_E4M3, m, h.FIT_SQ)
        P = int(gib * (1 << 30)) // (m * m)
        macs, popcs = gram_algorithmic_work(m)
        idx_np = np.sort(rng.choice(P, size=256, replace=False))
        ref = oracle.fitness(oracle.init_slots(m, idx_np, 2), oracle.FIT_SQ)
        rows = []
        for name, storage, path in M32_GRAM_PATHS:
            pop = h.empty_population(storage, m, P)
            fit = torch.zeros(P, dtype=torch.int32, device="cuda")
            h.ga_init_batch(pop, storage, m, P, 2)
            h.ga_fitness_batch(pop, storage, m, P, h.FIT_SQ, path, fit)
            torch.cuda.synchronize()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record()
            for _ in range(reps):
                h.ga_fitness_batch(pop, storage, m, P, h.FIT_SQ, path, fit)
            ev[1].record()
            ev[1].synchronize()
            sec = ev[0].elapsed_time(ev[1]) / 1e3 / reps
            got = fit.index_select(0, torch.as_tensor(idx_np, device="cuda")).cpu().numpy()
            exact = bool(np.array_equal(ref, got.view(np.uint32).astype(np.uint64)))
            nbytes = P * h.storage_bytes(storage, m)
            t_mem = nbytes / (hbm * 1e9)
            if storage == h.STORE_BITS:
                ops, peak, unit = P * popcs, popc_rate, "popc32"
            elif tuned_e4m3["path"] == h.PATH_FP8:   # AUTO on e4m3 resolved to tcgen05
                ops, peak, unit = P * macs, fp8_rate, "e4m3 MAC (tcgen05)"
            else:                                     # AUTO on e4m3 resolved to the warp-level FP8 MMA
                ops, peak, unit = P * macs, e4m3_warp_rate, "e4m3 MAC (mma.sync)"
            row = {"path": name, "ms": sec * 1e3, "matrices_per_s": P / sec, "exact_256_sampled": exact}
            if storage == h.STORE_E4M3:
                row["auto_resolved_to"] = {3: "tcgen05 FP8", 6: "FP8 mma.sync"}.get(tuned_e4m3["path"],
                                                                                 str(tuned_e4m3["path"]))
            row.update(_roof_entry(sec, t_mem, ops / peak, unit, peak, ops, nbytes, hbm))
            rows.append(row)
            del pop, fit
            torch.cuda.empty_cache()
        best = min(rows, key=lambda r: r["ms"])
        out.append({"m": m, "P": P, "paths": rows, "fastest": best["path"], "fastest_frac": best["frac"],
                    "fastest_bound": best["bound"]})
    return out


def m32_ga_report(dev, gens=500, call=100, prefix=50):
    """Config 5 in the default line: m = 100, P = 20,000 bit-packed balanced
    matrices (seed 4), F_sq, NC = NR = 1, `gens` generations of the fused
    path in ga_step calls of `call`, with full recomputation and with the
    incremental Gram-delta fitness (a GPU full recheck after every call).
    Checked against the oracle: the first `prefix` generations from the
    initial population, and one generation from the GPU's state after
    `gens` generations (population and fitness bit for bit, both modes).
    Roofline of each mode against its algorithmic work: offspring Gram
    popcounts (full: D ceil(m/32) per offspring; incremental: E[c(m-c)]
    ceil(m/32) cross dot products) and HBM bytes (P*S + 16P, plus the
    stored Gram read and written in incremental mode)."""
    import numpy as np
    import torch

    import oracle
    from paper_2208_14961_gb300 import hadga as h
    from paper_2208_14961_gb300 import peaks
    m, N, seed = 100, 5000, 4
    P = 4 * N
    stream = torch.cuda.Stream(device=dev)

    def fresh(inc):
        p = h.Population(m, N, seed=seed, fitness=h.FIT_SQ, storage=h.STORE_BITS, traj_cap=gens + 1,
                         stream=stream, device=dev)
        p.init_population()
        p.fitness()
        if inc:
            p.set_incremental(True)
        p.sync()
        return p

    w = fresh(True)
    w.step(call)
    w.sync()
    w.close()
    ref0 = oracle.init_population(m, P, seed, 0)
    F0 = oracle.fitness(ref0, oracle.FIT_SQ)
    refp, Fp = ref0.copy(), F0.copy()
    oracle.run(refp, Fp, N, 1, 1, oracle.FIT_SQ, seed, 0, 0, prefix)
    W = (m + 31) // 32
    D = (m - 1) * (m - 2) // 2
    cuts = range(1, m)
    e_cross = sum(c * (m - c) for c in cuts) / (m - 1)
    e_gram_read = sum((c * (c - 1) + (m - c) * (m - c - 1)) / 2 for c in cuts) / (m - 1)
    popc_rate = peaks.rate("popc_chain")
    hbm, hbm_kind = _peaks()
    base_bytes = bytes_per_generation(m, N)
    res, trajs = {}, {}
    for mode in ("full", "incremental"):
        inc = mode == "incremental"
        p = fresh(inc)
        p.step(prefix)
        p.sync()
        prefix_ok = bool(np.array_equal(p.as_int8(), refp)) and bool(np.array_equal(p.fitness_host(), Fp))
        p.close()
        p = fresh(inc)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms, checks, mism = 0.0, 0, 0
        for _ in range(gens // call):
            e0.record(stream)
            p.step(call)
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
            if inc:
                a, b = p.check_incremental()
                checks += 1
                mism += a + b
        trajs[mode] = p.trajectory()[0].astype(np.uint64)
        snap_pop, snap_F = p.as_int8(), p.fitness_host()
        p.step(1)
        p.sync()
        oracle.run(snap_pop, snap_F, N, 1, 1, oracle.FIT_SQ, seed, 0, gens, 1)
        step_ok = bool(np.array_equal(p.as_int8(), snap_pop)) and bool(np.array_equal(p.fitness_host(), snap_F))
        p.close()
        sec = ms / 1e3
        gps = gens / sec
        if inc:
            ops = 2 * N * e_cross * W
            nbytes = base_bytes + 2 * N * (e_gram_read + m * (m - 1) / 2)
            work = "offspring cross dot products E[c(m-c)] = %.0f x %d popc32 + stored Gram bytes" % (e_cross, W)
        else:
            ops = 2 * N * D * W
            nbytes = base_bytes
            work = "offspring Gram D x ceil(m/32) = %d x %d popc32 per offspring" % (D, W)
        t_gen = 1.0 / gps
        entry = {"generations": gens, "ms": ms, "generations_per_s": gps, "evals_per_s": gps * 2 * N,
                 "oracle_prefix_exact": prefix_ok, "oracle_step_exact_after": step_ok, "work": work}
        entry.update(_roof_entry(t_gen, nbytes / (hbm * 1e9), ops / popc_rate, "popc32", popc_rate, ops, nbytes,
                                 hbm))
        if inc:
            entry.update({"gpu_full_rechecks": checks, "recheck_mismatches": mism})
        res[mode] = entry
    res["incremental_over_full"] = res["incremental"]["generations_per_s"] / res["full"]["generations_per_s"]
    res["trajectories_equal"] = bool(np.array_equal(trajs["full"], trajs["incremental"]))
    res["workload"] = "m=100, P=20,000, bit storage, F_sq, NC=NR=1, seed 4"
    res["peaks"] = {"popc_per_s": popc_rate, "source": "measured (peaks microbenchmark)",
                    "hbm_gbs": hbm, "hbm_source": hbm_kind}
    return res


def m32plus_report(args, dev):
    """Orders m >= 32 (configs 3 and 5) for the default line: bounded to
    about a minute including the oracle checks."""
    from paper_2208_14961_gb300 import peaks
    t0 = time.perf_counter()
    hbm, hbm_kind = _peaks()
    popc_rate = peaks.rate("popc_chain")
    e4m3_warp = peaks.rate("mma_e4m3")
    fp8_rate, fp8_src = _fp8_mac_rate()
    ga = m32_ga_report(dev)
    gram = m32_gram_report(hbm, popc_rate, e4m3_warp, fp8_rate)
    return {"config5_ga_m100": ga, "config3_gram_8gib": gram,
            "peaks": {"hbm_gbs": hbm, "hbm_source": hbm_kind, "popc_per_s": popc_rate,
                      "mma_sync_e4m3_mac_per_s": e4m3_warp, "fp8_mac_per_s": fp8_rate, "fp8_source": fp8_src,
                      "note": "popc and mma.sync rates from the peaks microbenchmark"},
            "seconds": time.perf_counter() - t0}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-m32plus", action="store_true", help="skip the m >= 32 section of the default line")
    ap.add_argument("--plain-steps", type=int, default=4)
    ap.add_argument("--gram-sweep", action="store_true", help="precision sweep of the Gram + fitness paths")
    ap.add_argument("--gram-gb", type=float, default=8.0)
    ap.add_argument("--gram-ms", default="32,64,128,256")
    ap.add_argument("--gram-paths", default="")
    ap.add_argument("--mixed", action="store_true", help="mixed-order multi-population workload")
    ap.add_argument("--mixed-gens", type=int, default=500)
    ap.add_argument("--mixed-check", action="store_true")
    ap.add_argument("--mixed-compare-default", action="store_true",
                    help="also time the mixed workload with the default launch shapes")
    ap.add_argument("--incremental", action="store_true", help="incremental Gram-delta workload (m=100)")
    ap.add_argument("--inc-gens", type=int, default=10000)
    ap.add_argument("--table3", action="store_true", help="the paper's fitness-comparison workload (Sec. 4.2)")
    ap.add_argument("--t3-ms", default="20,40,60,80,100")
    ap.add_argument("--t3-gens", type=int, default=1000)
    ap.add_argument("--table1", action="store_true", help="the batched float Gram comparison of Sec. 2 (Table 1)")
    ap.add_argument("--t1-n", type=int, default=10000)
    ap.add_argument("--t1-m", type=int, default=100)
    ap.add_argument("--t1-reps", type=int, default=20)
    ap.add_argument("--t1-oracle-matrices", type=int, default=2000)
    ap.add_argument("--peaks", action="store_true", help="microbenchmark rates used by the roofline fractions")
    ap.add_argument("--search", action="store_true", help="time to a Hadamard matrix (the paper's Sec. 4.4 runs)")
    ap.add_argument("--search-ms", default="20,24,28")
    ap.add_argument("--search-seeds", type=int, default=3)
    ap.add_argument("--search-seconds", type=float, default=60.0)
    ap.add_argument("--search-chunk", type=int, default=2048)
    ap.add_argument("--table45", action="store_true", help="the paper's convergence tables (Sec. 4.3)")
    ap.add_argument("--t45-ms", default="12,16")
    ap.add_argument("--t45-seeds", type=int, default=20)
    ap.add_argument("--t45-cap", type=int, default=4000)
    ap.add_argument("--case", default="", help="one named small workload for ncu (see PROFILE_CASES)")
    ap.add_argument("--case-gens", type=int, default=8)
    args = ap.parse_args()
    if args.case:
        profile_case(args)
        return
    if args.peaks:
        peaks_report(args)
        return
    if args.gram_sweep:
        gram_sweep(args)
        return
    if args.mixed:
        mixed_workload(args)
        return
    if args.incremental:
        incremental_workload(args)
        return
    if args.table3:
        table3_workload(args)
        return
    if args.search:
        search_workload(args)
        return
    if args.table1:
        table1_workload(args)
        return
    if args.table45:
        table45_workload(args)
        return
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist

    from paper_2208_14961_gb300.build import build
    build()
    from paper_2208_14961_gb300 import hadga as h

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl" if dist.is_nccl_available() else "gloo")

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    stream = torch.cuda.Stream(device=dev)
    pop = h.Population(M, N, seed=SEED, pop_id=rank, NC=NC, NR=NR, fitness=h.FIT_SQ, storage=h.STORE_BITS,
                       traj_cap=STEP_GENS, device=dev, stream=stream)
    pop.init_population()
    pop.fitness()
    pop.sync()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)

    def flush_l2():
        with torch.cuda.stream(stream):
            flush.fill_(1)

    # ---- fused path, device-timed -------------------------------------------
    for _ in range(args.warmup):
        pop.step(STEP_GENS)
    pop.sync()
    pop.profile(True)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clock = ClockSampler(local)
    barrier()
    launches0 = h.kernel_launches()
    clock.start()
    for i in range(args.steps):
        flush_l2()
        starts[i].record(stream)
        pop.step(STEP_GENS)
        ends[i].record(stream)
    barrier()
    clocks = clock.stop()
    launches = h.kernel_launches() - launches0
    pop.sync()
    dev_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    perm_ms, fused_ms, fused_launches = pop.profile_read()
    pop.profile(False)
    gens = args.steps * STEP_GENS
    reduce_max = (lambda x: dist.all_reduce(x, op=dist.ReduceOp.MAX)) if world > 1 else None
    value, max_ms = job_rate(dev_ms / 1e3, gens, world, reduce_max, dev)
    max_ms *= 1e3

    # ---- plain path (one kernel per operator), device-timed ------------------
    pl = h.Population(M, N, seed=SEED, pop_id=rank, NC=NC, NR=NR, fitness=h.FIT_SQ, storage=h.STORE_BITS,
                      traj_cap=STEP_GENS, device=dev, stream=stream)
    pl.init_population()
    pl.fitness()
    pl.step_plain(STEP_GENS)
    pl.sync()
    plain_ms = 0.0
    for _ in range(args.plain_steps):
        flush_l2()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        pl.step_plain(STEP_GENS)
        b.record(stream)
        b.synchronize()
        plain_ms += a.elapsed_time(b)
    plain_gps = args.plain_steps * STEP_GENS / (plain_ms / 1e3)
    pl.close()

    # ---- end to end through the C ABI with host buffers ------------------------
    ee = h.Population(M, N, seed=SEED, pop_id=rank, NC=NC, NR=NR, fitness=h.FIT_SQ, storage=h.STORE_BITS,
                      traj_cap=STEP_GENS, device=dev, stream=stream)
    ee.init_population()
    ee.fitness()
    ee.sync()
    host_pop = ee.pop.cpu().pin_memory()
    host_fit = ee.fit.cpu().pin_memory()
    out_pop = torch.empty_like(host_pop).pin_memory()
    out_fit = torch.empty_like(host_fit).pin_memory()
    h2d = host_pop.numel() * host_pop.element_size() + host_fit.numel() * host_fit.element_size()
    # device -> host per step: the final population and fitness, the step's
    # best-fitness trajectory (ga_trajectory copies one 64-bit key per
    # generation) and the 4-byte device error word its synchronisation reads
    d2h = (out_pop.numel() * out_pop.element_size() + out_fit.numel() * out_fit.element_size()
           + STEP_GENS * 8 + 4)

    def e2e_step():
        with torch.cuda.stream(stream):
            ee.pop.copy_(host_pop, non_blocking=True)
            ee.fit.copy_(host_fit, non_blocking=True)
        ee.step(STEP_GENS)
        with torch.cuda.stream(stream):
            out_pop.copy_(ee.pop, non_blocking=True)
            out_fit.copy_(ee.fit, non_blocking=True)
        ee.trajectory()          # synchronises the stream: the step's results are on the host

    for _ in range(2):
        e2e_step()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_value, _ = job_rate(e2e_s, args.steps * STEP_GENS, world, reduce_max, dev)
    ee.close()

    # ---- roofline of the persistent kernel --------------------------------------
    peak, peak_kind = _peaks()
    roof = None
    if fused_launches > 0 and fused_ms > 0:
        per_launch_ms = fused_ms / fused_launches
        gens_per_launch = gens / fused_launches
        per_launch_bytes = bytes_per_generation() * gens_per_launch
        achieved = per_launch_bytes / (per_launch_ms / 1e3) / 1e9
        fresh = FUSED_M20_TRAFFIC["sources_sha256"] == fused_sources_sha256()
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": FUSED_M20_TRAFFIC["bytes"] if fresh else None,
                "traffic_note": ("ncu DRAM read+write of one launch of %d generations after a cache flush"
                                 % FUSED_M20_TRAFFIC["generations_per_launch"]) if fresh else
                                "kernel sources changed since the last capture",
                "kernel": "k_fused", "peak_source": peak_kind,
                "algorithmic_bytes_per_generation": bytes_per_generation(),
                "impl_bytes_per_generation": impl_bytes_per_generation(),
                "generations_per_launch": gens_per_launch,
                "launch_ms": per_launch_ms, "perm_table_ms_per_launch": perm_ms / max(fused_launches, 1)}

    # what binds instead of HBM: the two grid barriers of every generation
    sync = None
    try:
        from paper_2208_14961_gb300 import peaks
        bps = peaks.rate("grid_barriers")
        if bps > 0 and fused_launches > 0:
            gen_us = fused_ms / gens * 1e3
            sync = {"grid_barrier_us": 1e6 / bps, "barriers_per_generation": 2, "generation_us": gen_us,
                    "barrier_share": 2e6 / bps / gen_us,
                    "note": "grid barrier latency from the peaks microbenchmark (same barrier code, 152 blocks)"}
    except Exception as e:  # the context field must not break the bench line
        sync = {"error": str(e)[:200]}

    m32 = None
    if world == 1 and not args.no_m32plus:
        try:  # the m >= 32 context must not break the headline line
            m32 = m32plus_report(args, dev)
        except Exception as e:
            m32 = {"error": f"{type(e).__name__}: {e}"[:300]}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        gps, ngen, dt, cores = oracle_sample()
        cpu = {"value": gps, "unit": "generations/s", "cores": cores, "kind": "oracle",
               "sample": f"{ngen} generations of the same workload in {dt:.1f} s"}
        try:  # the single-core figure is context: it must not break the bench line
            gps1, ngen1, dt1, _ = oracle_sample(seconds=4.0, min_gens=2, threads=1)
            cpu["one_core"] = {"value": gps1, "sample": f"{ngen1} generations in {dt1:.1f} s on 1 thread"}
        except Exception as e:
            cpu["one_core"] = {"error": str(e)[:200]}

    if rank == 0:
        line = {
            "metric": METRIC, "arm": "fused persistent generation kernel",
            "value": value, "unit": "generations/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "generations_per_step": STEP_GENS, "storage": "bits",
                       "global_batch": P * world, "parallelism": f"replicas{world}",
                       "l2": "flushed before every step (256 MiB write), outside the timed events",
                       "fused": bool(pop.is_fused())},
            "evals_per_s": value * (P // 2),
            "evals_per_s_paper_convention": value * P,
            "plain": {"value": plain_gps, "unit": "generations/s", "steps": args.plain_steps,
                      "fused_over_plain": value / world / plain_gps},
            "e2e": {"value": e2e_value, "unit": "generations/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "roofline": roof,
            "sync_bound": sync,
            "m32plus": m32,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "gpu_launches": int(launches),
        }
        print(json.dumps(line), flush=True)
    pop.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
