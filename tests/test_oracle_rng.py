"""Pins of the oracle's random-number layer (CPU only)."""
import itertools
import math

import numpy as np
import pytest

import oracle
from hadamard_fixtures import philox_kat


@pytest.mark.parametrize("case", range(3))
def test_philox_known_answers(case):
    ctr, key, expect = philox_kat()[case]
    assert [int(x) for x in oracle.philox4x32_10(ctr, key)] == expect


def test_uniform_mapping_edges():
    # floor(w * span / 2^32): w = 0 gives lo, w = 2^32 - 1 gives hi.
    assert oracle.uniform(0, 1, 19) == 1
    assert oracle.uniform(0xFFFFFFFF, 1, 19) == 19
    assert oracle.uniform(0xFFFFFFFF, 0, 0) == 0
    # exact boundaries for span 3: w < 2^32/3 -> lo.
    assert oracle.uniform(1431655765, 0, 2) == 0
    assert oracle.uniform(1431655766, 0, 2) == 1
    for w in [0, 1, 12345, 2**31, 2**32 - 1]:
        for lo, hi in [(0, 0), (0, 11), (1, 255), (7, 4507)]:
            v = oracle.uniform(w, lo, hi)
            assert lo <= v <= hi
            assert v == lo + (w * (hi - lo + 1) >> 32)


def test_stream_is_consecutive_philox_blocks():
    seed, pop_id, op, gen, index, sub = 7, 3, oracle.OP_MUTATE, 11, 42, 5
    words = oracle.stream_words(seed, pop_id, op, gen, index, sub, 10)
    for b in range(3):
        blk = oracle.philox4x32_10([op, gen, index, (sub << 16) | b], [seed, pop_id])
        got = words[4 * b:4 * b + 4]
        assert list(got) == list(blk[:len(got)])


def test_select_keys_are_stream_words():
    """u_d is word d mod 4 of Philox block (SELECT, gen, d // 4, 0)."""
    for d in range(12):
        blk = oracle.philox4x32_10([oracle.OP_SELECT, 5, d // 4, 0], [9, 2])
        assert oracle.select_key(9, 2, 5, d) == int(blk[d % 4])


@pytest.mark.parametrize("n", [1, 2, 3, 8, 33, 1000, 20000])
def test_perm_is_argsort_of_keys(n):
    keys = [oracle.select_key(4, 1, 7, d) for d in range(n)]
    expect = sorted(range(n), key=lambda d: (keys[d], d))
    assert list(oracle.perm(n, 4, 1, 7)) == expect


@pytest.mark.parametrize("n", [3, 4, 5])
def test_perm_uniform_over_orders(n):
    """Chi-square over all n! orders across many (seed, generation) keys."""
    counts = {}
    k = math.factorial(n)
    trials = 200 * k
    for t in range(trials):
        perm = tuple(int(x) for x in oracle.perm(n, t, 1, 9))
        counts[perm] = counts.get(perm, 0) + 1
    assert len(counts) == k
    expect = trials / k
    chi2 = sum((c - expect) ** 2 / expect for c in counts.values())
    # 99.9% quantiles of chi-square with k - 1 = 5, 23, 119 degrees of freedom
    assert chi2 < {3: 20.5, 4: 49.7, 5: 173.6}[n], chi2


def test_perm_depends_on_generation_and_key():
    n = 64
    a = list(oracle.perm(n, 1, 0, 1))
    assert a != list(oracle.perm(n, 1, 0, 2))
    assert a != list(oracle.perm(n, 2, 0, 1))
    assert a != list(oracle.perm(n, 1, 1, 1))


def test_mixed_order_sizes_in_range():
    Ns = [oracle.mixed_N(3, i) for i in range(7)]
    assert all(500 <= N <= 5000 for N in Ns)
    assert len(set(Ns)) > 1


@pytest.mark.parametrize("seed", [3, 0, 77])
def test_mixed_order_sizes_from_the_config_stream(seed):
    """N of order position idx is 500 + U[0, 4500] of word 0 of the Philox
    block with key (seed, 0) and counter (CONFIG, generation 0, idx, 0),
    rebuilt here from the known-answer-pinned Philox and the multiply-shift
    map lo + floor(w (hi - lo + 1) / 2^32): a wrong key, op, index or span
    fails it."""
    for idx in range(7):
        w0 = int(oracle.philox4x32_10([oracle.OP_CONFIG, 0, idx, 0], [seed, 0])[0])
        assert oracle.mixed_N(seed, idx) == 500 + ((w0 * 4501) >> 32)
