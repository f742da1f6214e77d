"""Pins of the oracle's truncation selection and survivor placement."""
import numpy as np
import pytest

import oracle
from inputs import random_pm1


@pytest.mark.parametrize("N,seed", [(1, 0), (2, 1), (5, 2), (16, 3), (50, 4)])
def test_survivors_brute_force(N, seed):
    rng = np.random.default_rng(seed)
    P = 4 * N
    F = rng.integers(0, 6, P).astype(np.uint64)     # many ties on purpose
    ranked = sorted(range(P), key=lambda q: (int(F[q]), q))
    expect = sorted(ranked[:2 * N])
    assert list(oracle.survivors(F, N)) == expect


@pytest.mark.parametrize("N,gen", [(1, 1), (3, 2), (8, 5), (25, 7)])
def test_select_brute_force(N, gen):
    m, seed, pop_id = 8, 13, 2
    P = 4 * N
    pop = random_pm1(P, m, seed=N)
    rng = np.random.default_rng(gen)
    F = rng.integers(0, 10, P).astype(np.uint64)
    old_pop, old_F = pop.copy(), F.copy()
    oracle.select(pop, F, N, seed, pop_id, gen)
    ranked = sorted(range(P), key=lambda q: (int(old_F[q]), q))
    surv = sorted(ranked[:2 * N])
    keys = [oracle.select_key(seed, pop_id, gen, d) for d in range(2 * N)]
    pi = sorted(range(2 * N), key=lambda d: (keys[d], d))
    for p in range(2 * N):
        assert np.array_equal(pop[p], old_pop[surv[pi[p]]])
        assert F[p] == old_F[surv[pi[p]]]
    assert np.array_equal(pop[2 * N:], old_pop[2 * N:])   # offspring slots untouched
    # the multiset of surviving fitness values is the 2N smallest
    assert sorted(F[:2 * N].tolist()) == sorted(old_F.tolist())[:2 * N]


def test_best_lowest_slot_on_ties():
    F = np.array([5, 3, 9, 3, 3], dtype=np.uint64)
    assert oracle.best(F) == (1, 3)
