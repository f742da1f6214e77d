"""Named small workloads for profiling one kernel at a time.

  python -m paper_2208_14961_gb300.cases <case> [generations]

fused_m20   m=20, P=40,000, bit storage: init, fitness, then `generations`
            (default 8) generations in one persistent launch
plain_m20   the same with the one-kernel-per-operator path
inc_m100    m=100, P=20,000, bit storage, incremental Gram-delta fitness:
            init, fitness, Gram store, then `generations` generations
full_m100   the same workload with full fitness recomputation
gram_m<M>_<path>  Gram + fitness of a population of ~1 GiB (int8 size) at
            order M with path int32 | imma | popc8 | popc | fp8 | bf16 | fp8w
real_<f32|f64>_m<M>  batched real Gram Q^T Q of 10,000 uniform random
            matrices of order M (two launches)
"""
import sys

import torch

from paper_2208_14961_gb300.build import build


def main(argv):
    build()
    from paper_2208_14961_gb300 import hadga as h
    case = argv[0]
    gens = int(argv[1]) if len(argv) > 1 else 8
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
    raise SystemExit(f"unknown case {case}")


if __name__ == "__main__":
    main(sys.argv[1:])
