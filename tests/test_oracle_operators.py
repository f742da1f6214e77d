"""Pins of the oracle's init, crossover and mutation (CPU only)."""
import itertools

import numpy as np
import pytest

import oracle
from hadamard_fixtures import crossover_fig2, mutation_fig3
from inputs import balanced_pm1, random_pm1


def test_crossover_worked_example_fig2():
    cut, mats = crossover_fig2()
    O1, O2 = oracle.crossover_pair(mats["P1"], mats["P2"], cut)
    assert np.array_equal(O1, mats["O1"])
    assert np.array_equal(O2, mats["O2"])


@pytest.mark.parametrize("part", ["a", "b", "c", "d"])
def test_mutation_worked_example_fig3(part):
    ex = mutation_fig3()[part]
    M = ex["matrix"]
    assert np.all(M[:, 0] == 1) and np.all(M.sum(axis=0)[1:] == 0)
    Q = M.copy()
    r1 = [p[0] for p in ex["pairs"]]
    r2 = [p[1] for p in ex["pairs"]]
    flips = oracle.mutate_explicit(Q, ex["cols"], r1, r2)
    changed = {(int(i), int(j)) for i, j in zip(*np.nonzero(Q != M))}
    assert changed == ex["success"]
    assert flips == len(ex["success"]) // 2
    assert not (changed & ex["fail"])
    # per-column successes quoted by the figure / prose
    per_col = {c: sum(1 for (_, j) in ex["success"] if j == c) // 2 for c in ex["cols"]}
    expect = {"a": {6: 2, 5: 1, 2: 0}, "b": {5: 1, 2: 0, 4: 2},
              "c": {3: 1, 1: 1, 6: 0}, "d": {2: 1, 7: 2, 6: 1}}[part]
    assert per_col == expect


def test_mutation_fig3a_printed_indices_disagree():
    """The printed index rows of part (a) do not reproduce its figure."""
    ex = mutation_fig3()["a"]
    Q = ex["matrix"].copy()
    r1 = [p[0] for p in ex["printed_pairs"]]
    r2 = [p[1] for p in ex["printed_pairs"]]
    oracle.mutate_explicit(Q, ex["cols"], r1, r2)
    changed = {(int(i), int(j)) for i, j in zip(*np.nonzero(Q != ex["matrix"]))}
    assert changed != ex["success"]


def test_mutation_sequential_semantics_with_repeats():
    """A repeated column re-applies the same pairs and undoes the flips."""
    Q = balanced_pm1(1, 12, seed=1)[0]
    M = Q.copy()
    n = oracle.mutate_explicit(Q, [5, 5], [0, 3], [1, 7])
    assert np.array_equal(Q, M) and n % 2 == 0
    # pairs sharing a row: order matters
    Q = np.ones((4, 4), np.int8)
    Q[:, 1] = [-1, 1, 1, -1]
    oracle.mutate_explicit(Q, [1], [0, 1], [1, 2])
    # (0,1): -1,+1 -> flip -> +1,-1 ; (1,2): -1,+1 -> flip -> +1,-1
    assert list(Q[:, 1]) == [1, 1, -1, -1]


@pytest.mark.parametrize("m,c", [(4, 1), (12, 5), (20, 19), (32, 16)])
def test_crossover_conserves_columns(m, c):
    P1, P2 = random_pm1(2, m, seed=m + c)
    O1, O2 = oracle.crossover_pair(P1, P2, c)
    for j in range(m):
        pair_in = sorted([tuple(P1[:, j]), tuple(P2[:, j])])
        pair_out = sorted([tuple(O1[:, j]), tuple(O2[:, j])])
        assert pair_in == pair_out
    assert np.array_equal(O1[:, :c], P1[:, :c]) and np.array_equal(O1[:, c:], P2[:, c:])


def test_cut_points_and_draws_in_range():
    m = 20
    cuts = [oracle.cut_point(m, 1, 0, 3, k) for k in range(2000)]
    assert min(cuts) == 1 and max(cuts) == m - 1
    for o in range(200):
        c, r1, r2 = oracle.mutation_draws(m, 3, 4, 1, 0, 3, o)
        assert np.all((c >= 1) & (c <= m - 1))
        assert np.all((r1 >= 0) & (r1 < m)) and np.all((r2 >= 0) & (r2 < m))
    # the stream order: NC columns, then NR first rows, then NR second rows
    w = oracle.stream_words(1, 0, oracle.OP_MUTATE, 3, 7, 0, 11)
    c, r1, r2 = oracle.mutation_draws(m, 3, 4, 1, 0, 3, 7)
    assert list(c) == [1 + (int(x) * (m - 1) >> 32) for x in w[:3]]
    assert list(r1) == [int(x) * m >> 32 for x in w[3:7]]
    assert list(r2) == [int(x) * m >> 32 for x in w[7:11]]


@pytest.mark.parametrize("m,NC,NR", [(12, 1, 1), (20, 4, 2), (32, 3, 6)])
def test_mutation_population_invariants(m, NC, NR):
    N = 40
    pop = oracle.init_population(m, 4 * N, seed=2)
    before = pop.copy()
    oracle.mutate(pop, N, NC, NR, seed=2, pop_id=0, gen=1)
    assert np.array_equal(pop[:2 * N], before[:2 * N])           # parents untouched
    assert np.all(pop[:, :, 0] == 1)
    assert np.all(pop.astype(np.int32).sum(axis=1)[:, 1:] == 0)   # balance kept
    changed = (pop != before).reshape(4 * N, -1).sum(axis=1)
    assert np.all(changed <= 2 * NC * NR) and changed.sum() > 0


@pytest.mark.parametrize("m", [4, 12, 20, 100])
def test_init_balance_and_first_column(m):
    pop = oracle.init_population(m, 64, seed=0)
    assert np.all(pop[:, :, 0] == 1)
    assert np.all(pop.astype(np.int32).sum(axis=1)[:, 1:] == 0)
    if m >= 12:   # order 4 has only 216 such matrices, so repeats are expected
        assert len({pop[i].tobytes() for i in range(64)}) == 64


def test_init_uniform_over_balanced_columns_m4():
    """Chi-square: each of the 6 balanced columns of order 4 equally likely."""
    pop = oracle.init_population(4, 3000, seed=11)
    cols = pop[:, :, 1:].transpose(0, 2, 1).reshape(-1, 4)
    keys, counts = np.unique(cols, axis=0, return_counts=True)
    assert len(keys) == 6
    expect = cols.shape[0] / 6
    chi2 = float(((counts - expect) ** 2 / expect).sum())
    assert chi2 < 20.5   # 99.9% quantile, 5 dof


def test_init_slots_equal_those_of_the_whole_population():
    pop = oracle.init_population(24, 50, seed=3, pop_id=2)
    idx = [0, 7, 31, 49]
    assert np.array_equal(oracle.init_slots(24, idx, 3, 2), pop[idx])


def test_init_deterministic_and_thread_independent():
    a = oracle.init_population(20, 100, seed=1)
    n0 = oracle.num_threads()
    oracle.set_num_threads(1)
    b = oracle.init_population(20, 100, seed=1)
    oracle.set_num_threads(n0)
    c = oracle.init_population(20, 100, seed=2)
    d = oracle.init_population(20, 100, seed=1, pop_id=1)
    assert np.array_equal(a, b) and not np.array_equal(a, c) and not np.array_equal(a, d)


def test_init_follows_fisher_yates_on_the_stream():
    """Slot 3, column 2 of order 8 rebuilt from the raw stream words."""
    m, seed, slot, j = 8, 9, 3, 2
    w = oracle.stream_words(seed, 0, oracle.OP_INIT, 0, slot, j, m - 1)
    v = [-1] * (m // 2) + [1] * (m // 2)
    for i1 in range(m - 1):
        i2 = i1 + (int(w[i1]) * (m - i1) >> 32)
        v[i1], v[i2] = v[i2], v[i1]
    pop = oracle.init_population(m, 4, seed)
    assert list(pop[slot, :, j]) == v


@pytest.mark.parametrize("m,N", [(8, 9), (12, 25), (20, 40)])
def test_mutation_method1_one_draw_for_the_generation(m, N):
    """Sec. 3.5, method 1: the same column and the same two rows for every
    offspring of a generation, a pair switched only where its signs differ.
    Checked from the definition: the flips of all offspring lie on one
    column and one row pair, every offspring whose two entries differ there
    is switched and every other one is unchanged, and the column and rows
    are the first three words of stream (MUTATE, gen, 2N) mapped to
    [1, m-1], [0, m-1], [0, m-1]."""
    seed, pop_id, gen = 6, 1, 3
    pop = oracle.init_population(m, 4 * N, seed, pop_id)
    oracle.crossover(pop, N, seed, pop_id, gen)
    before = pop.copy()
    oracle.mutate(pop, N, 1, 1, seed, pop_id, gen, shared=1)
    w = oracle.stream_words(seed, pop_id, oracle.OP_MUTATE, gen, 2 * N, 0, 3)
    col = 1 + (int(w[0]) * (m - 1) >> 32)
    r1 = int(w[1]) * m >> 32
    r2 = int(w[2]) * m >> 32
    assert np.array_equal(pop[:2 * N], before[:2 * N])
    switched = 0
    for o in range(2 * N, 4 * N):
        a, b = before[o, r1, col], before[o, r2, col]
        expect = before[o].copy()
        if a != b:
            expect[r1, col], expect[r2, col] = -a, -b
            switched += 1
        assert np.array_equal(pop[o], expect), o
    assert switched > 0 or r1 == r2


def test_mutation_method1_run_differs_from_method2():
    """The two methods draw from different streams: same start, different
    populations after a generation (and both keep every column balanced)."""
    m, N, seed = 12, 30, 2
    a = oracle.init_population(m, 4 * N, seed)
    b = a.copy()
    Fa = oracle.fitness(a, oracle.FIT_SQ)
    Fb = Fa.copy()
    oracle.run(a, Fa, N, 1, 1, oracle.FIT_SQ, seed, 0, 0, 3, shared_mutation=0)
    oracle.run(b, Fb, N, 1, 1, oracle.FIT_SQ, seed, 0, 0, 3, shared_mutation=1)
    assert not np.array_equal(a, b)
    for pop in (a, b):
        assert np.all(pop[:, :, 0] == 1)
        assert np.all(pop[:, :, 1:].sum(axis=1) == 0)
