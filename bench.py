"""Throughput of the GA population step on GB300 (one JSON line on stdout).

Workload: m = 20, P = 40,000 balanced +-1 matrices (N = 10,000; the paper's
stated scale), fitness = sum over i < j of G_ij^2, one balanced pair-flip per
child (NC = NR = 1), Philox seed 1, bit storage.  A step is one chunk of
STEP_GENS generations of the whole hot path (selection, survivor placement,
crossover, mutation, offspring fitness, best individual), run by the fused
persistent generation kernel through the C ABI (ga_step).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

value     generations/s of the fused path, inputs resident in HBM, CUDA events
          on the context's stream; the L2 cache is flushed (256 MiB write)
          before every step, outside the timed events.
e2e       the same metric with the population and fitness copied in from
          pinned host memory and the step's best-fitness trajectory copied
          back, every step, inside the timed region (wall clock).
plain     the one-kernel-per-operator path on the same workload.
roofline  the persistent kernel against the measured HBM copy bandwidth.
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
STEP_GENS = 50
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


# DRAM read + write bytes of one k_fused launch of this workload from the
# ncu capture summarised in profiles/k_fused_m20_P40k.md (the population
# stays in L2 across the generations of a launch, so the cold read of the
# starting population is the whole traffic and does not grow with the
# generations per launch).
FUSED_M20_DRAM_BYTES_PER_LAUNCH = 3.464448e6


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
    """Algorithmic HBM bytes of one generation of the fused kernel (bit
    storage): read the 2N surviving parents, write all 4N slots (2N parents
    placed + 2N offspring), read and write the 4N fitness words, read the
    survivor-order row (2N words)."""
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
                 "--format=csv,noheader,nounits", "-lms", "200"],
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
    blocks = autotune.tune_fused_grid(specs, stream=stream)

    def fresh():
        pops = []
        for i, (m, N) in enumerate(specs):
            p = h.Population(m, N, seed=3, pop_id=i, fitness=h.FIT_SQ, storage=h.STORE_BITS, traj_cap=512,
                             stream=stream)
            p.init_population()
            p.fitness()
            pops.append(p)
        h.set_fused_grid(pops[0], blocks)
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
            "P": [4 * N for _, N in specs], "generations": gens, "graph_chunk": chunk, "autotuned_blocks": blocks,
            "ms": ms, "generations_per_s": gens / (ms / 1e3),
            "evals_per_s": gens * (total_P // 2) / (ms / 1e3), "exact_vs_oracle": exact}
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
                  (28, 10_000, 1, 10, 428_082, 3_054)]


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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--plain-steps", type=int, default=4)
    ap.add_argument("--gram-sweep", action="store_true", help="precision sweep of the Gram + fitness paths")
    ap.add_argument("--gram-gb", type=float, default=8.0)
    ap.add_argument("--gram-ms", default="32,64,128,256")
    ap.add_argument("--gram-paths", default="")
    ap.add_argument("--mixed", action="store_true", help="mixed-order multi-population workload")
    ap.add_argument("--mixed-gens", type=int, default=500)
    ap.add_argument("--mixed-check", action="store_true")
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
    args = ap.parse_args()
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
    h2d = host_pop.numel() * host_pop.element_size() + host_fit.numel() * host_fit.element_size()
    d2h = STEP_GENS * 8          # the step's best-fitness trajectory (one 64-bit key per generation)
    for _ in range(2):
        with torch.cuda.stream(stream):
            ee.pop.copy_(host_pop, non_blocking=True)
            ee.fit.copy_(host_fit, non_blocking=True)
        ee.step(STEP_GENS)
        ee.trajectory()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            ee.pop.copy_(host_pop, non_blocking=True)
            ee.fit.copy_(host_fit, non_blocking=True)
        ee.step(STEP_GENS)
        ee.trajectory()          # device -> host read of the step's result
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_value, _ = job_rate(e2e_s, args.steps * STEP_GENS, world, reduce_max, dev)
    ee.close()

    # ---- roofline of the persistent kernel --------------------------------------
    peak, peak_kind = _peaks()
    roof = None
    if fused_launches > 0 and fused_ms > 0:
        per_launch_ms = fused_ms / fused_launches
        per_launch_bytes = bytes_per_generation() * STEP_GENS
        achieved = per_launch_bytes / (per_launch_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": FUSED_M20_DRAM_BYTES_PER_LAUNCH, "kernel": "k_fused", "peak_source": peak_kind,
                "launch_ms": per_launch_ms, "perm_table_ms_per_launch": perm_ms / max(fused_launches, 1)}

    # what binds instead of HBM: the two grid barriers of every generation
    sync = None
    try:
        from paper_2208_14961_gb300 import peaks
        bps = peaks.rate("grid_barriers")
        if bps > 0 and fused_launches > 0:
            gen_us = fused_ms / fused_launches / STEP_GENS * 1e3
            sync = {"grid_barrier_us": 1e6 / bps, "barriers_per_generation": 2, "generation_us": gen_us,
                    "barrier_share": 2e6 / bps / gen_us,
                    "note": "grid barrier latency from the peaks microbenchmark (same barrier code, 152 blocks)"}
    except Exception as e:  # the context field must not break the bench line
        sync = {"error": str(e)[:200]}

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
