"""GPU parity of the incremental Gram-delta mode (a7) against the oracle.

The incremental path keeps every individual's Gram and updates it by the
column-exchange block rule and the O(m) pair-flip rule; its populations,
fitness values, trajectories and stored Gram matrices must equal the
oracle's full recomputation exactly."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def _oracle(m, N, seed, gens, NC=1, NR=1, kind=0, pop_id=0):
    ref = oracle.init_population(m, 4 * N, seed, pop_id)
    F = oracle.fitness(ref, kind)
    _, tf, ts = oracle.run(ref, F, N, NC, NR, kind, seed, pop_id, 0, gens)
    return ref, F, tf, ts


def _gpu(h, m, N, seed, gens, NC=1, NR=1, kind=0, pop_id=0, graph=False):
    pop = h.Population(m, N, seed=seed, pop_id=pop_id, NC=NC, NR=NR, fitness=kind, storage=1,
                       traj_cap=max(gens, 1), stream=torch.cuda.Stream() if graph else None)
    pop.init_population()
    pop.fitness()
    pop.set_incremental(True)
    if graph:
        h.step_multi_graph([pop], gens, chunk=10)
    else:
        pop.step(gens)
    pop.sync()
    return pop


@pytest.mark.parametrize("m,N,NC,NR,kind", [(36, 25, 1, 1, 0), (36, 40, 2, 3, 1), (64, 30, 1, 1, 0),
                                            (64, 20, 3, 2, 2), (100, 20, 1, 1, 0), (100, 16, 2, 4, 1),
                                            (128, 12, 1, 1, 0), (44, 33, 1, 10, 2),
                                            (68, 21, 1, 1, 0), (92, 19, 2, 2, 2)])
def test_incremental_matches_oracle(m, N, NC, NR, kind):
    h = need_gpu()
    gens = 30
    pop = _gpu(h, m, N, 11, gens, NC, NR, kind, pop_id=2)
    rp, rF, tf, ts = _oracle(m, N, 11, gens, NC, NR, kind, pop_id=2)
    assert np.array_equal(pop.fitness_host(), rF)
    assert np.array_equal(pop.as_int8(), rp)
    gtf, gts = pop.trajectory()
    assert np.array_equal(gtf.astype(np.uint64), tf)
    assert np.array_equal(gts, ts)
    assert pop.check_incremental() == (0, 0)
    # the stored Gram of some slots (parents and offspring) is the oracle's
    for slot in (0, N, 2 * N, 3 * N, 4 * N - 1):
        assert np.array_equal(pop.gram(slot), oracle.gram(rp[slot]).astype(np.int32)), slot
    pop.close()


def test_incremental_graph_replay_and_resume():
    """Graph replay of chunks, a stretch of plain operators (which marks the
    Gram storage stale), and fused generations again equal one oracle run."""
    h = need_gpu()
    m, N, seed = 100, 24, 5
    pop = _gpu(h, m, N, seed, 20, graph=True)
    assert pop.check_incremental() == (0, 0)
    pop.step_plain(3)
    pop.step(7)
    pop.sync()
    rp, rF, tf, ts = _oracle(m, N, seed, 30)
    assert np.array_equal(pop.fitness_host(), rF)
    assert np.array_equal(pop.as_int8(), rp)
    assert pop.check_incremental() == (0, 0)
    pop.close()


def test_incremental_odd_chunks_and_reenable():
    """Generation counts that end on the second ping-pong buffer, and a
    population replaced from the host (the Gram storage is rebuilt)."""
    h = need_gpu()
    m, N, seed = 64, 50, 3
    pop = _gpu(h, m, N, seed, 67)
    assert pop.check_incremental() == (0, 0)
    pop.step(1)
    pop.sync()
    rp, rF, _, _ = _oracle(m, N, seed, 68)
    assert np.array_equal(pop.fitness_host(), rF)
    assert np.array_equal(pop.as_int8(), rp)
    # replace the population by a fresh one and continue from generation 0
    fresh = oracle.init_population(m, 4 * N, 99, 0)
    pop.load_int8(fresh)
    pop.set_generation(0)
    pop.fitness()
    pop.step(5)
    pop.sync()
    F0 = oracle.fitness(fresh, 0)
    oracle.run(fresh, F0, N, 1, 1, 0, seed, 0, 0, 5)
    assert np.array_equal(pop.as_int8(), fresh)
    assert np.array_equal(pop.fitness_host(), F0)
    assert pop.check_incremental() == (0, 0)
    pop.set_incremental(False)
    pop.close()


def test_incremental_rejects_unsupported_contexts():
    h = need_gpu()
    for m, storage in ((20, 1), (64, 0), (132, 1)):
        pop = h.Population(m, 8, seed=0, storage=storage)
        with pytest.raises(h.GAError):
            pop.set_incremental(True)
        pop.close()
    pop = h.Population(64, 8, seed=0, storage=1)
    with pytest.raises(h.GAError):
        pop.check_incremental()  # mode off
    pop.close()


def test_incremental_with_mutation_method1():
    """The incremental Gram path under mutation method 1 (the same flipped
    column in every offspring of a generation)."""
    h = need_gpu()
    m, N, seed, gens = 64, 30, 9, 25
    pop = h.Population(m, N, seed=seed, fitness=0, storage=1, traj_cap=gens, mutation=1)
    pop.init_population()
    pop.fitness()
    pop.set_incremental(True)
    pop.step(gens)
    pop.sync()
    ref = oracle.init_population(m, 4 * N, seed)
    F = oracle.fitness(ref, 0)
    oracle.run(ref, F, N, 1, 1, 0, seed, 0, 0, gens, shared_mutation=1)
    assert np.array_equal(pop.as_int8(), ref)
    assert np.array_equal(pop.fitness_host(), F)
    assert pop.check_incremental() == (0, 0)
    pop.close()


@pytest.mark.parametrize("m,N", [(64, 600), (100, 300)])
def test_auto_choice_measures_both_and_leaves_the_state(m, N):
    """ga_set_incremental(AUTO) times both modes from the current population,
    keeps the faster, and leaves population, fitness, generation and
    trajectory as they were; the run that follows matches the oracle."""
    h = need_gpu()
    gens0, gens = 5, 8
    pop = h.Population(m, N, seed=6, storage=h.STORE_BITS, traj_cap=64)
    pop.init_population()
    pop.fitness()
    pop.step(gens0)
    pop.sync()
    before = pop.as_int8(), pop.fitness_host(), pop.trajectory(), pop.generation()
    pop.set_incremental("auto")
    on, full_ms, inc_ms = pop.incremental_choice()
    assert full_ms > 0 and inc_ms > 0
    assert on == (inc_ms < full_ms)
    after = pop.as_int8(), pop.fitness_host(), pop.trajectory(), pop.generation()
    assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
    assert np.array_equal(before[2][0], after[2][0]) and np.array_equal(before[2][1], after[2][1])
    assert before[3] == after[3] == gens0
    pop.step(gens)
    pop.sync()
    ref = oracle.init_population(m, 4 * N, 6)
    F = oracle.fitness(ref, oracle.FIT_SQ)
    oracle.run(ref, F, N, 1, 1, oracle.FIT_SQ, 6, 0, 0, gens0 + gens)
    assert np.array_equal(pop.as_int8(), ref) and np.array_equal(pop.fitness_host(), F)
    if on:
        assert pop.check_incremental() == (0, 0)
    pop.close()


@pytest.mark.parametrize("incremental", [False, True])
def test_config5_full_size_prefix(incremental):
    """Config 5 at its real size (m = 100, P = 20,000, bit storage, F_sq,
    NC = NR = 1, seed 4): 20 generations of the fused path, with full
    recomputation or the incremental Gram-delta fitness, equal to the oracle;
    the incremental state passes a GPU full recheck."""
    h = need_gpu()
    m, N, gens = 100, 5000, 20
    pop = h.Population(m, N, seed=4, storage=h.STORE_BITS, traj_cap=gens)
    pop.set_strict(True)
    pop.init_population()
    pop.fitness()
    if incremental:
        pop.set_incremental(True)
    pop.step(gens)
    pop.sync()
    ref = oracle.init_population(m, 4 * N, 4)
    F = oracle.fitness(ref, oracle.FIT_SQ)
    _, tf, ts = oracle.run(ref, F, N, 1, 1, oracle.FIT_SQ, 4, 0, 0, gens)
    assert np.array_equal(pop.as_int8(), ref) and np.array_equal(pop.fitness_host(), F)
    gtf, gts = pop.trajectory()
    assert np.array_equal(gtf.astype(np.uint64), tf) and np.array_equal(gts, ts)
    if incremental:
        assert pop.check_incremental() == (0, 0)
    pop.close()
