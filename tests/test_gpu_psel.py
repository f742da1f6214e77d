"""GPU parity of the probabilistic selection (the Sec. 3.3 variant with
probabilities inverse to the fitness; weights floor(2^32 / (F + 1))):
whole generations of the one-kernel-per-operator path and of the fused
persistent kernel against the oracle's generation loop, bit for bit."""
import numpy as np
import pytest

import oracle
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def _gpu(h, m, N, seed, gens, storage, mode, NC=1, NR=1, kind=0, strict=False):
    pop = h.Population(m, N, seed=seed, NC=NC, NR=NR, fitness=kind, storage=storage, traj_cap=max(gens, 1),
                       selection=h.SEL_PROBABILISTIC)
    if strict:
        pop.set_strict(True)
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


def _oracle(m, N, seed, gens, NC=1, NR=1, kind=0):
    ref = oracle.init_population(m, 4 * N, seed)
    F = oracle.fitness(ref, kind)
    _, tf, ts = oracle.run(ref, F, N, NC, NR, kind, seed, 0, 0, gens, selection=oracle.SEL_PROBABILISTIC)
    return ref, F, tf, ts


def _same(gpu, ref):
    p, F, (gtf, gts) = gpu
    rp, rF, tf, ts = ref
    assert np.array_equal(F, rF)
    assert np.array_equal(p, rp)
    assert np.array_equal(gtf.astype(np.uint64), tf)
    assert np.array_equal(gts, ts)


@pytest.mark.parametrize("mode", ["plain", "fused"])
@pytest.mark.parametrize("storage", [0, 1])
def test_m12_P1000_matches_oracle(mode, storage):
    h = need_gpu()
    _same(_gpu(h, 12, 250, 0, 40, storage, mode, strict=mode == "fused"), _oracle(12, 250, 0, 40))


@pytest.mark.parametrize("mode", ["plain", "fused"])
@pytest.mark.parametrize("m,N,NC,NR,kind,gens", [(4, 1, 1, 1, 0, 6), (20, 63, 2, 3, 2, 15), (32, 100, 1, 1, 1, 10),
                                                  (40, 37, 1, 2, 0, 8), (100, 20, 3, 1, 2, 5),
                                                  (128, 9, 1, 1, 0, 4)])
def test_orders_ragged_populations_and_fitness_kinds(mode, m, N, NC, NR, kind, gens):
    """Both build paths of the fused kernel (m <= 32 four threads per pair,
    m > 32 a warp per offspring), a population that is not a multiple of 32
    (ragged last tile, whose slots past P weigh nothing), NC / NR > 1, F1, F2."""
    h = need_gpu()
    _same(_gpu(h, m, N, 7, gens, 1, mode, NC, NR, kind, strict=mode == "fused"),
          _oracle(m, N, 7, gens, NC, NR, kind))


def test_fused_m20_P40000_prefix():
    """The paper's scale (m = 20, P = 40,000), 12 generations."""
    h = need_gpu()
    _same(_gpu(h, 20, 10000, 1, 12, 1, "fused", strict=True), _oracle(20, 10000, 1, 12))


def test_fused_large_population():
    """2N = 60,000 parents drawn by weight (no survivor-order table)."""
    h = need_gpu()
    _same(_gpu(h, 16, 30000, 3, 5, 1, "fused", strict=True), _oracle(16, 30000, 3, 5))


def test_probabilistic_selection_refuses_incremental_mode():
    h = need_gpu()
    pop = h.Population(64, 16, seed=1, storage=h.STORE_BITS, selection=h.SEL_PROBABILISTIC)
    with pytest.raises(h.GAError) as ei:
        pop.set_incremental(True)
    assert ei.value.status == h.GA_EUNSUPPORTED
    pop.close()


def test_mixed_selection_methods_in_one_multi_step():
    """Populations with different selection methods cannot share one
    persistent launch: ga_step_multi runs them one by one (and strict
    contexts report GA_EUNSUPPORTED)."""
    h = need_gpu()
    m, N, gens = 12, 40, 6
    pops = []
    for i, sel in enumerate((h.SEL_TRUNCATION, h.SEL_PROBABILISTIC)):
        p = h.Population(m, N, seed=2, pop_id=i, storage=h.STORE_BITS, traj_cap=gens, selection=sel)
        p.init_population()
        p.fitness()
        pops.append(p)
    h.step_multi(pops, gens)
    for i, (sel, p) in enumerate(zip((0, 1), pops)):
        p.sync()
        ref = oracle.init_population(m, 4 * N, 2, i)
        F = oracle.fitness(ref, 0)
        oracle.run(ref, F, N, 1, 1, 0, 2, i, 0, gens, selection=sel)
        assert np.array_equal(p.as_int8(), ref) and np.array_equal(p.fitness_host(), F)
    pops[0].set_strict(True)
    with pytest.raises(h.GAError) as ei:
        h.step_multi(pops, 1)
    assert ei.value.status == h.GA_EUNSUPPORTED
    for p in pops:
        p.close()
