"""GPU parity of whole generations (plain operators and the fused
persistent kernel) against the oracle's generation loop."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def _run_gpu(h, m, N, seed, gens, storage, mode, NC=1, NR=1, kind=0, pop_id=0):
    pop = h.Population(m, N, seed=seed, pop_id=pop_id, NC=NC, NR=NR, fitness=kind, storage=storage,
                       traj_cap=max(gens, 1))
    pop.init_population()
    pop.fitness()
    if mode == "plain":
        pop.step_plain(gens)
    else:
        pop.step(gens)
    pop.sync()
    out = pop.as_int8(), pop.fitness_host(), pop.trajectory()
    pop.close()
    return out


def _run_oracle(m, N, seed, gens, NC=1, NR=1, kind=0, pop_id=0):
    ref = oracle.init_population(m, 4 * N, seed, pop_id)
    F = oracle.fitness(ref, kind)
    _, tf, ts = oracle.run(ref, F, N, NC, NR, kind, seed, pop_id, 0, gens)
    return ref, F, tf, ts


def _assert_same(gpu, ref):
    p, F, (gtf, gts) = gpu
    rp, rF, tf, ts = ref
    assert np.array_equal(F, rF)
    assert np.array_equal(p, rp)
    assert np.array_equal(gtf.astype(np.uint64), tf)
    assert np.array_equal(gts, ts)


@pytest.mark.parametrize("mode", ["plain", "fused"])
@pytest.mark.parametrize("storage", [0, 1])
def test_config1_m12_P1000_200_generations(mode, storage):
    """m = 12, P = 1,000, F_sq, one pair-flip per child, 200 generations, seed 0."""
    h = need_gpu()
    _assert_same(_run_gpu(h, 12, 250, 0, 200, storage, mode), _run_oracle(12, 250, 0, 200))


@pytest.mark.parametrize("mode", ["plain", "fused"])
def test_config2_m20_P40000_prefix(mode):
    """m = 20, P = 40,000 (the paper's scale), seed 1: the first 25 generations."""
    h = need_gpu()
    _assert_same(_run_gpu(h, 20, 10000, 1, 25, 1, mode), _run_oracle(20, 10000, 1, 25))


@pytest.mark.parametrize("mode", ["plain", "fused"])
@pytest.mark.parametrize("m,N,NC,NR,kind", [(4, 1, 1, 1, 0), (8, 3, 2, 2, 2), (16, 40, 4, 2, 1),
                                            (28, 33, 1, 10, 2), (36, 25, 2, 3, 0), (100, 20, 1, 1, 0)])
def test_small_configs(mode, m, N, NC, NR, kind):
    h = need_gpu()
    _assert_same(_run_gpu(h, m, N, 7, 30, 1, mode, NC, NR, kind, pop_id=3),
                 _run_oracle(m, N, 7, 30, NC, NR, kind, pop_id=3))
