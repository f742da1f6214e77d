"""Pins of the oracle's probabilistic selection (Sec. 3.3: probabilities
inverse proportional to the fitness; the weights floor(2^32 / (F + 1)) and
the 64-bit draws are this build's reading of that sentence).  Each pin is
independent of the oracle's own arithmetic: hand-written interval tables on
tiny weights, the equal-weight case reducing to a textbook multiply-shift of
raw (known-answer pinned) Philox words, chi-square against w / W, the
degenerate and monotone cases, and the copy invariants of a whole
selection."""
import math

import numpy as np
import pytest

import oracle

TWO31 = 1 << 31


def _u64(seed, pop_id, gen, p):
    w = oracle.philox4x32_10([oracle.OP_PSELECT, gen, p, 0], [seed, pop_id])
    return (int(w[0]) << 32) | int(w[1])


def test_weights_at_small_fitness():
    # 2^32 / (F + 1) for F = 0, 1, 2, 3, 15 and the F ~ 2^31 end where weights are 1 or 2
    assert [oracle.psel_weight(f) for f in (0, 1, 2, 3, 15)] == [4294967296, 2147483648, 1431655765,
                                                                  1073741824, 268435456]
    assert oracle.psel_weight(TWO31) == 1 and oracle.psel_weight(TWO31 - 1) == 2


def test_interval_table_on_tiny_weights():
    """Weights (1, 2, 1): W = 4 and t = floor(u * 4 / 2^64) in {0, 1, 2, 3};
    by the definition t = 0 picks individual 0, t = 1, 2 individual 1, t = 3
    individual 2 (the table is written out here, not computed)."""
    F = np.array([TWO31, TWO31 - 1, TWO31], dtype=np.uint64)   # weights 1, 2, 1
    table = {0: 0, 1: 1, 2: 1, 3: 2}
    seen = set()
    for gen in range(1, 200):
        for p in range(2):
            t = (_u64(7, 0, gen, p) * 4) >> 64
            seen.add(t)
            assert oracle.psel_pick(F, 7, 0, gen, p) == table[t]
    assert seen == {0, 1, 2, 3}


def test_equal_weights_reduce_to_multiply_shift():
    """All weights 1: the pick is the 64-bit multiply-shift floor(u P / 2^64)
    of the raw Philox words (Lemire's map, no rejection)."""
    P = 12
    F = np.full(P, TWO31, dtype=np.uint64)
    for gen in (1, 2, 99):
        for p in range(6):
            assert oracle.psel_pick(F, 3, 1, gen, p) == (_u64(3, 1, gen, p) * P) >> 64


def _chi2_pvalue(obs, probs):
    n = sum(obs)
    stat = sum((o - n * q) ** 2 / (n * q) for o, q in zip(obs, probs))
    k = len(obs) - 1
    # Wilson-Hilferty normal approximation of the chi-square tail
    z = ((stat / k) ** (1 / 3) - (1 - 2 / (9 * k))) / math.sqrt(2 / (9 * k))
    return 0.5 * math.erfc(z / math.sqrt(2))


def test_frequencies_follow_inverse_fitness():
    """F = (0, 1, 3, 7): weights 2^32, 2^31, 2^30, 2^29, i.e. probabilities
    8/15, 4/15, 2/15, 1/15; 20,000 draws."""
    F = np.array([0, 1, 3, 7], dtype=np.uint64)
    C = np.cumsum([oracle.psel_weight(int(f)) for f in F]).astype(np.uint64)
    counts = [0] * 4
    for gen in range(1, 10001):
        for p in range(2):
            counts[oracle.psel_pick(F, 11, 0, gen, p)] += 1
    assert _chi2_pvalue(counts, [8 / 15, 4 / 15, 2 / 15, 1 / 15]) > 1e-4
    assert int(C[-1]) == 15 * (1 << 29)


def test_equal_fitness_is_uniform():
    F = np.full(6, 5, dtype=np.uint64)
    counts = [0] * 6
    for gen in range(1, 6001):
        for p in range(2):
            counts[oracle.psel_pick(F, 2, 0, gen, p)] += 1
    assert _chi2_pvalue(counts, [1 / 6] * 6) > 1e-4


def test_a_hadamard_matrix_is_almost_always_chosen():
    """F = (0, 2^31, 2^31, 2^31): weights 2^32, 1, 1, 1; any other pick has
    probability 3 / (2^32 + 3)."""
    F = np.array([0, TWO31, TWO31, TWO31], dtype=np.uint64)
    assert all(oracle.psel_pick(F, 5, 0, g, p) == 0 for g in range(1, 3001) for p in range(2))


def test_lower_fitness_is_chosen_more_often():
    F = np.array([10, 20, 40, 80, 160], dtype=np.uint64)
    counts = [0] * 5
    for gen in range(1, 8001):
        for p in range(2):
            counts[oracle.psel_pick(F, 4, 2, gen, p)] += 1
    assert counts == sorted(counts, reverse=True)


def test_whole_selection_copies_the_drawn_individuals():
    m, N, seed, gen = 8, 6, 13, 4
    pop = oracle.init_population(m, 4 * N, seed)
    F = oracle.fitness(pop, oracle.FIT_SQ)
    before_pop, before_F = pop.copy(), F.copy()
    oracle.select_prob(pop, F, N, seed, 0, gen)
    for p in range(2 * N):
        q = oracle.psel_pick(before_F, seed, 0, gen, p)
        assert np.array_equal(pop[p], before_pop[q]) and F[p] == before_F[q]
    # the offspring half is left for crossover to overwrite
    assert np.array_equal(pop[2 * N:], before_pop[2 * N:]) and np.array_equal(F[2 * N:], before_F[2 * N:])


def test_run_with_probabilistic_selection_keeps_the_invariants():
    m, N, gens = 12, 25, 10
    pop = oracle.init_population(m, 4 * N, 1)
    F = oracle.fitness(pop, oracle.FIT_SQ)
    n, tf, ts = oracle.run(pop, F, N, 1, 1, oracle.FIT_SQ, 1, 0, 0, gens, selection=oracle.SEL_PROBABILISTIC)
    assert n == gens
    assert np.array_equal(F, oracle.fitness(pop, oracle.FIT_SQ))
    assert np.all(pop[:, :, 0] == 1)                          # column 0 stays +1
    assert np.all(pop.sum(axis=1)[:, 1:] == 0)                # balanced columns
    # differs from truncation selection on the same start
    pop2 = oracle.init_population(m, 4 * N, 1)
    F2 = oracle.fitness(pop2, oracle.FIT_SQ)
    oracle.run(pop2, F2, N, 1, 1, oracle.FIT_SQ, 1, 0, 0, gens)
    assert not np.array_equal(pop, pop2)
