"""Pins of the oracle's Gram and fitness functions (CPU only)."""
import itertools

import numpy as np
import pytest

import oracle
from hadamard_fixtures import paley1, sylvester
from inputs import balanced_pm1, random_pm1

KINDS = [oracle.FIT_SQ, oracle.FIT_ABS, oracle.FIT_NNZ]


@pytest.mark.parametrize("m", [4, 8, 16, 32, 64, 128, 256])
def test_sylvester_is_optimal(m):
    H = sylvester(m)
    assert np.all(H[:, 0] == 1)
    for kind in KINDS:
        assert int(oracle.fitness(H[None], kind)[0]) == 0


@pytest.mark.parametrize("q", [11, 19, 23, 31, 43, 47])
def test_paley_is_optimal(q):
    H = paley1(q)
    m = q + 1
    # independent check that the fixture is Hadamard
    assert np.array_equal(H.astype(np.int64).T @ H.astype(np.int64), m * np.eye(m, dtype=np.int64))
    for kind in KINDS:
        assert int(oracle.fitness(H[None], kind)[0]) == 0


def test_kronecker_of_hadamard_is_optimal():
    H = np.kron(paley1(11), sylvester(2)).astype(np.int8)  # order 24
    H = (H * H[:, :1]).astype(np.int8)
    for kind in KINDS:
        assert int(oracle.fitness(H[None], kind)[0]) == 0


@pytest.mark.parametrize("m", [12, 20, 24, 32])
def test_single_flip_closed_form(m):
    """One successful pair flip in a Hadamard matrix: F2 = m - 2,
    F1 = 4m - 8, F_sq = 8m - 16 (rows of a Hadamard matrix differ in m/2
    columns, so m/2 - 1 entries of one Gram row move to +-4)."""
    H = sylvester(m) if m in (32,) else paley1(m - 1)
    rng = np.random.default_rng(m)
    for _ in range(20):
        Q = H.copy()
        c = int(rng.integers(1, m))
        while True:
            r1, r2 = (int(x) for x in rng.integers(0, m, 2))
            if Q[r1, c] != Q[r2, c]:
                break
        Q[r1, c] = -Q[r1, c]
        Q[r2, c] = -Q[r2, c]
        F = {k: int(oracle.fitness(Q[None], k)[0]) for k in KINDS}
        assert F[oracle.FIT_NNZ] == m - 2
        assert F[oracle.FIT_ABS] == 4 * m - 8
        assert F[oracle.FIT_SQ] == 8 * m - 16


def test_m4_enumeration():
    """All 216 matrices with column 0 = +1 and balanced columns 1..3."""
    bal = [np.array(v, np.int8) for v in itertools.product([-1, 1], repeat=4) if sum(v) == 0]
    assert len(bal) == 6
    pops = []
    for a, b, c in itertools.product(range(6), repeat=3):
        Q = np.ones((4, 4), np.int8)
        Q[:, 1], Q[:, 2], Q[:, 3] = bal[a], bal[b], bal[c]
        pops.append(Q)
    pop = np.stack(pops)
    F2 = oracle.fitness(pop, oracle.FIT_NNZ)
    Fsq = oracle.fitness(pop, oracle.FIT_SQ)
    u2, c2 = np.unique(F2, return_counts=True)
    us, cs = np.unique(Fsq, return_counts=True)
    assert dict(zip(u2.tolist(), c2.tolist())) == {0: 48, 2: 144, 6: 24}
    assert dict(zip(us.tolist(), cs.tolist())) == {0: 48, 16: 144, 48: 24}
    # the 48 optimal ones are exactly the Hadamard ones
    is_h = np.array([np.array_equal(Q.astype(int).T @ Q.astype(int), 4 * np.eye(4)) for Q in pop])
    assert np.array_equal(is_h, F2 == 0)


@pytest.mark.parametrize("m", [4, 12, 20, 36])
def test_gram_matches_float64_matmul(m):
    pop = random_pm1(6, m, seed=m)
    for Q in pop:
        G = oracle.gram(Q)
        Gf = Q.astype(np.float64).T @ Q.astype(np.float64)
        assert np.array_equal(G, Gf.astype(np.int32))
        assert np.array_equal(G, G.T) and np.all(np.diag(G) == m)


@pytest.mark.parametrize("m", [8, 12, 20, 64])
def test_fitness_definitions_against_float64_gram(m):
    pop = random_pm1(10, m, seed=100 + m)
    G = np.einsum("pri,prj->pij", pop.astype(np.float64), pop.astype(np.float64))
    iu = np.triu_indices(m, 1)
    sq = (G[:, iu[0], iu[1]] ** 2).sum(axis=1)
    ab = np.abs(G).sum(axis=(1, 2)) - m * m
    nz = (G != 0).sum(axis=(1, 2)) - m
    assert np.array_equal(oracle.fitness(pop, oracle.FIT_SQ), sq.astype(np.uint64))
    assert np.array_equal(oracle.fitness(pop, oracle.FIT_ABS), ab.astype(np.uint64))
    assert np.array_equal(oracle.fitness(pop, oracle.FIT_NNZ), nz.astype(np.uint64))


@pytest.mark.parametrize("m", [12, 20, 32])
def test_fsq_row_gram_identity(m):
    """F_sq = (||Q Q^T||_F^2 - m^3) / 2: a row-Gram computation that shares
    nothing with the column Gram."""
    pop = random_pm1(8, m, seed=7 * m)
    R = np.einsum("pik,pjk->pij", pop.astype(np.int64), pop.astype(np.int64))
    expect = ((R ** 2).sum(axis=(1, 2)) - m ** 3) // 2
    assert np.array_equal(oracle.fitness(pop, oracle.FIT_SQ), expect.astype(np.uint64))


@pytest.mark.parametrize("m", [8, 12, 20, 28])
def test_balanced_invariants(m):
    pop = balanced_pm1(50, m, seed=m)
    for Q in pop[:5]:
        G = oracle.gram(Q)
        assert np.all(G[0, 1:] == 0)           # balanced columns are orthogonal to column 0
        assert np.all(G % 4 == 0)              # m = 0 mod 4 and balanced columns
    assert np.all(oracle.fitness(pop, oracle.FIT_SQ) % 16 == 0)
    assert np.all(oracle.fitness(pop, oracle.FIT_ABS) % 8 == 0)
    assert np.all(oracle.fitness(pop, oracle.FIT_NNZ) % 2 == 0)


@pytest.mark.parametrize("m", [12, 20])
def test_fitness_invariant_under_symmetries(m):
    pop = balanced_pm1(4, m, seed=3 * m)
    rng = np.random.default_rng(0)
    for Q in pop:
        base = {k: int(oracle.fitness(Q[None], k)[0]) for k in KINDS}
        perm = np.concatenate([[0], 1 + rng.permutation(m - 1)])
        sign = np.concatenate([[1], rng.choice([-1, 1], m - 1)]).astype(np.int8)
        rows = rng.permutation(m)
        Q2 = np.ascontiguousarray((Q[:, perm] * sign)[rows])
        for k in KINDS:
            assert int(oracle.fitness(Q2[None], k)[0]) == base[k]


def test_fitness_range_and_thread_independence():
    pop = random_pm1(64, 20, seed=5)
    a = oracle.fitness(pop, oracle.FIT_SQ)
    n0 = oracle.num_threads()
    oracle.set_num_threads(1)
    b = oracle.fitness(pop, oracle.FIT_SQ)
    oracle.set_num_threads(n0)
    assert np.array_equal(a, b)
    part = np.zeros(64, np.uint64)
    oracle.fitness(pop, oracle.FIT_SQ, first=10, count=20, out=part)
    assert np.array_equal(part[10:30], a[10:30]) and not part[:10].any() and not part[30:].any()
