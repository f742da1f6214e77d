"""The two Gram update rules the incremental fitness mode (a7) relies on,
checked against the oracle's full Gram on random populations (CPU only).

Pair flip: flipping Q[r1][c] = s and Q[r2][c] = -s changes only row and
column c of G = Q^T Q, entry (c, j) by -2s(Q[r1][j] - Q[r2][j]).
Column exchange at cut c: the offspring's G keeps the top parent's block
G[:c, :c] and the bottom parent's block G[c:, c:]; only the c(m - c) cross
entries are new."""
import numpy as np

import oracle


def test_pair_flip_changes_only_row_and_column_c():
    rng = np.random.default_rng(5)
    for m in (12, 20, 36, 64):
        pop = oracle.init_population(m, 8, 3, 0)
        for Q in pop:
            G = oracle.gram(Q).astype(np.int64)
            c = int(rng.integers(1, m))
            col = Q[:, c]
            r1 = int(rng.choice(np.flatnonzero(col == 1)))
            r2 = int(rng.choice(np.flatnonzero(col == -1)))
            s = int(Q[r1, c])
            Q2 = Q.copy()
            Q2[r1, c] *= -1
            Q2[r2, c] *= -1
            G2 = oracle.gram(Q2).astype(np.int64)
            delta = -2 * s * (Q[r1, :].astype(np.int64) - Q[r2, :].astype(np.int64))
            expect = G.copy()
            for j in range(m):
                if j != c:
                    expect[c, j] += delta[j]
                    expect[j, c] += delta[j]
            assert np.array_equal(G2, expect)
            changed = np.argwhere(G2 != G)
            assert all(i == c or j == c for i, j in changed)
            assert set(np.unique(G2 - G)) <= {-4, 0, 4}


def test_column_exchange_keeps_the_parents_blocks():
    for m in (12, 36, 100):
        pop = oracle.init_population(m, 4, 8, 1)
        P1, P2 = pop[0], pop[1]
        G1, G2 = oracle.gram(P1), oracle.gram(P2)
        for c in (1, m // 3, m - 1):
            O1, O2 = oracle.crossover_pair(P1, P2, c)
            GO1, GO2 = oracle.gram(O1), oracle.gram(O2)
            assert np.array_equal(GO1[:c, :c], G1[:c, :c])
            assert np.array_equal(GO1[c:, c:], G2[c:, c:])
            assert np.array_equal(GO2[:c, :c], G2[:c, :c])
            assert np.array_equal(GO2[c:, c:], G1[c:, c:])
            X = P1[:, :c].astype(np.int64).T @ P2[:, c:].astype(np.int64)
            assert np.array_equal(GO1[:c, c:], X)

