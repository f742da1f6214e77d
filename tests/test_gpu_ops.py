"""GPU parity of the individual operators against the oracle, through the
C ABI: init, Gram + fitness on every path, selection, crossover, mutation,
storage conversion.  Integer results must be bit-exact."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import fit_u64, need_gpu, to_device_int8
from hadamard_fixtures import paley1, sylvester
from inputs import balanced_pm1, random_pm1

pytestmark = pytest.mark.gpu

KINDS = [0, 1, 2]


@pytest.mark.parametrize("m", [4, 12, 20, 32, 36, 100, 256])
@pytest.mark.parametrize("storage", [0, 1, 2, 3])
def test_init_matches_oracle(m, storage):
    h = need_gpu()
    P = 37 if m <= 36 else 9   # ragged: not a multiple of 4 or 32
    seed, pop_id = 5, 2
    pop = h.empty_population(storage, m, P)
    h.ga_init_batch(pop, storage, m, P, seed, pop_id)
    out = h.empty_population(0, m, P)
    h.ga_convert(pop, storage, out, 0, m, P)
    torch.cuda.synchronize()
    ref = oracle.init_population(m, P, seed, pop_id)
    assert np.array_equal(out.cpu().numpy(), ref)


@pytest.mark.parametrize("m", [4, 8, 12, 16, 20, 24, 28, 32, 36, 64, 100, 128, 256])
@pytest.mark.parametrize("path,storage", [(5, 1), (5, 0), (1, 0), (2, 0), (6, 2)])
def test_fitness_paths_match_oracle(m, path, storage):
    h = need_gpu()
    P = 45 if m <= 64 else 11
    host = np.concatenate([random_pm1(P - 5, m, seed=m), balanced_pm1(5, m, seed=m + 1)])
    src = to_device_int8(host)
    pop = h.empty_population(storage, m, P)
    h.ga_convert(src, 0, pop, storage, m, P)
    for kind in KINDS:
        fit = torch.zeros(P, dtype=torch.int32, device="cuda")
        h.ga_fitness_batch(pop, storage, m, P, kind, path, fit)
        assert np.array_equal(fit_u64(fit), oracle.fitness(host, kind)), (m, path, storage, kind)


@pytest.mark.parametrize("m", [68, 96, 132, 200, 252])
@pytest.mark.parametrize("storage", [1, 0])
def test_popc_word_counts_match_oracle(m, storage):
    """Column widths W = 3, 5, 7 and 8 words: the carry-save population
    count takes the tree's partial levels there."""
    h = need_gpu()
    P = 9
    host = np.concatenate([random_pm1(P - 3, m, seed=m), balanced_pm1(3, m, seed=m + 1)])
    src = to_device_int8(host)
    pop = h.empty_population(storage, m, P)
    h.ga_convert(src, 0, pop, storage, m, P)
    for kind in KINDS:
        fit = torch.zeros(P, dtype=torch.int32, device="cuda")
        h.ga_fitness_batch(pop, storage, m, P, kind, 5, fit)
        assert np.array_equal(fit_u64(fit), oracle.fitness(host, kind)), (m, storage, kind)


@pytest.mark.parametrize("path,storage", [(5, 1), (5, 0), (1, 0), (2, 0), (6, 2)])
def test_known_hadamard_matrices_score_zero(path, storage):
    h = need_gpu()
    mats = [sylvester(m) for m in (4, 8, 16, 32, 64, 128, 256)] + [paley1(q) for q in (11, 19, 23, 43)]
    for H in mats:
        m = H.shape[0]
        src = to_device_int8(H[None])
        pop = h.empty_population(storage, m, 1)
        h.ga_convert(src, 0, pop, storage, m, 1)
        for kind in KINDS:
            fit = torch.full((1,), 7, dtype=torch.int32, device="cuda")
            h.ga_fitness_batch(pop, storage, m, 1, kind, path, fit)
            assert int(fit_u64(fit)[0]) == 0, (m, kind)


@pytest.mark.parametrize("src_st,dst_st", [(0, 1), (1, 0), (0, 2), (2, 3), (3, 1), (1, 2)])
def test_convert_round_trip(src_st, dst_st):
    h = need_gpu()
    m, P = 36, 13
    host = random_pm1(P, m, seed=3)
    a = h.empty_population(src_st, m, P)
    h.ga_convert(to_device_int8(host), 0, a, src_st, m, P)
    b = h.empty_population(dst_st, m, P)
    h.ga_convert(a, src_st, b, dst_st, m, P)
    c = h.empty_population(0, m, P)
    h.ga_convert(b, dst_st, c, 0, m, P)
    torch.cuda.synchronize()
    assert np.array_equal(c.cpu().numpy(), host)


def _fresh(h, m, N, seed, storage, NC=1, NR=1, kind=0, path=0):
    pop = h.Population(m, N, seed=seed, NC=NC, NR=NR, fitness=kind, storage=storage, path=path)
    pop.init_population()
    pop.fitness()
    return pop


@pytest.mark.parametrize("m,N", [(4, 1), (4, 9), (12, 250), (20, 300), (36, 40), (100, 12), (256, 3),
                                 (4, 12288), (20, 12287)])
@pytest.mark.parametrize("storage", [0, 1])
def test_select_matches_oracle(m, N, storage):
    """Includes the largest shared-memory survivor sort (2N = 24,576) and a
    ragged one (2N = 24,574, not a multiple of the four keys per draw)."""
    h = need_gpu()
    seed = 11
    pop = _fresh(h, m, N, seed, storage)
    ref = oracle.init_population(m, 4 * N, seed)
    refF = oracle.fitness(ref, 0)
    assert np.array_equal(pop.fitness_host(), refF)
    for g in (1, 2):
        pop.select()
        oracle.select(ref, refF, N, seed, 0, g)
        assert pop.generation() == g
        assert np.array_equal(pop.as_int8(), ref)
        assert np.array_equal(pop.fitness_host(), refF)
    pop.sync()


def test_select_with_heavy_ties_and_large_population():
    """m = 4 has three fitness values only; 2N = 32768 exceeds the
    shared-memory survivor sort and takes the global-memory one."""
    h = need_gpu()
    m, N, seed = 4, 16384, 3
    pop = _fresh(h, m, N, seed, 1)
    ref = oracle.init_population(m, 4 * N, seed)
    refF = oracle.fitness(ref, 0)
    pop.select()
    oracle.select(ref, refF, N, seed, 0, 1)
    assert np.array_equal(pop.as_int8(), ref)
    assert np.array_equal(pop.fitness_host(), refF)


@pytest.mark.parametrize("m,N,NC,NR", [(12, 50, 1, 1), (20, 64, 4, 2), (36, 17, 3, 5), (100, 6, 2, 2),
                                       (8, 10, 64, 64)])
@pytest.mark.parametrize("storage", [0, 1])
def test_crossover_and_mutation_match_oracle(m, N, NC, NR, storage):
    h = need_gpu()
    seed = 21
    pop = _fresh(h, m, N, seed, storage, NC=NC, NR=NR)
    ref = oracle.init_population(m, 4 * N, seed)
    pop.set_generation(4)
    pop.crossover()
    oracle.crossover(ref, N, seed, 0, 4)
    assert np.array_equal(pop.as_int8(), ref)
    pop.mutate()
    oracle.mutate(ref, N, NC, NR, seed, 0, 4)
    assert np.array_equal(pop.as_int8(), ref)


def test_set_get_slot_and_best():
    h = need_gpu()
    m, N = 12, 10
    pop = _fresh(h, m, N, 1, 1)
    H = paley1(11)
    pop.set_slot(17, H)
    assert np.array_equal(pop.get_slot(17), H)
    pop.fitness()
    assert pop.best() == (17, 0)


@pytest.mark.parametrize("m", [32, 64, 128, 256])
def test_config3_full_size_sampled(m):
    """The precision sweep's workload at full size: P = 8 GiB / m^2 balanced
    matrices (seed 2), every Gram path on its own storage, the launch shapes
    the sweep times; 48 seeded slots checked against the oracle one by one
    (the oracle builds those slots' initial matrices itself; the device init
    writes the same content in every storage)."""
    h = need_gpu()
    P = (8 << 30) // (m * m)
    rng = np.random.default_rng(m)
    idx = np.sort(rng.choice(P, size=48, replace=False))
    sample = oracle.init_slots(m, idx, 2)
    expected = oracle.fitness(sample, oracle.FIT_SQ)
    for path, storage in ((1, 0), (2, 0), (5, 0), (5, 1), (3, 2), (6, 2), (4, 3)):
        pop = h.empty_population(storage, m, P)
        h.ga_init_batch(pop, storage, m, P, 2)
        fit = torch.zeros(P, dtype=torch.int32, device="cuda")
        h.ga_fitness_batch(pop, storage, m, P, 0, path, fit)
        got = fit.index_select(0, torch.as_tensor(idx, device="cuda")).cpu().numpy().view(np.uint32)
        assert np.array_equal(got.astype(np.uint64), expected), (m, path, storage)
        del pop, fit
        torch.cuda.empty_cache()


@pytest.mark.parametrize("m,P", [(36, 100_000), (128, 80_000), (200, 80_000)])
@pytest.mark.parametrize("storage", [0, 1])
def test_popc_warps_with_several_matrices(m, P, storage):
    """Populations larger than the grid's warps (8 x 64 blocks x 152 SMs =
    77,824), so warps take a second matrix; sampled slots from both rounds."""
    h = need_gpu()
    rng = np.random.default_rng(m + 7)
    split = 77_824
    idx = np.sort(np.concatenate([rng.choice(split, 16, replace=False),
                                  rng.choice(np.arange(split, P), 32, replace=False), [P - 1]]))
    sample = oracle.init_slots(m, idx, 5)
    pop = h.empty_population(storage, m, P)
    h.ga_init_batch(pop, storage, m, P, 5)
    tidx = torch.as_tensor(idx, device="cuda")
    for kind in KINDS:
        fit = torch.zeros(P, dtype=torch.int32, device="cuda")
        h.ga_fitness_batch(pop, storage, m, P, kind, 5, fit)
        got = fit.index_select(0, tidx).cpu().numpy().view(np.uint32).astype(np.uint64)
        assert np.array_equal(got, oracle.fitness(sample, kind)), (m, storage, kind)


def test_empty_batches_are_no_ops():
    h = need_gpu()
    for storage in (0, 1, 2, 3):
        pop = h.empty_population(storage, 32, 1)
        fit = torch.full((1,), 7, dtype=torch.int32, device="cuda")
        h.ga_init_batch(pop, storage, 32, 0, 1)
        h.ga_fitness_batch(pop, storage, 32, 0, 0, 0, fit)
        torch.cuda.synchronize()
        assert int(fit[0]) == 7
