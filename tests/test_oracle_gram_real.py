"""Pins of the oracle's batched real Gram F_b = Q_b^T Q_b (Sec. 2, Table 1)
against closed forms and exact arithmetic, independent of its own loop."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from hadamard_fixtures import sylvester
from inputs import signed_real, uniform_real

U64 = 2.0 ** -53


def gamma(n: int, u: float) -> float:
    """Bound on the relative error of an n-term recursive sum of products
    (Higham, Accuracy and Stability of Numerical Algorithms, Sec. 3.1)."""
    return n * u / (1.0 - n * u)


@pytest.mark.parametrize("m", [1, 2, 4, 8, 16, 32, 64])
def test_sylvester_gives_m_times_identity(m):
    H = sylvester(m).astype(np.float64)
    assert np.array_equal(oracle.gram_real(H), m * np.eye(m))


def test_diagonal_squares_its_entries():
    d = np.random.default_rng(1).random(7) * 4 - 2
    G = oracle.gram_real(np.diag(d))
    assert np.array_equal(G, np.diag(d * d))


@pytest.mark.parametrize("r,c", [(0, 3), (4, 1), (2, 2)])
def test_single_entry_lands_on_its_column(r, c):
    """Q with one nonzero x at (r, c): Q^T Q has x^2 at (c, c) and nothing
    else; the row index r must not appear (Q Q^T would put it at (r, r))."""
    Q = np.zeros((5, 5))
    Q[r, c] = 3.0
    G = oracle.gram_real(Q)
    E = np.zeros((5, 5))
    E[c, c] = 9.0
    assert np.array_equal(G, E)


def test_rank_one_closed_form():
    """Q = u v^T gives Q^T Q = (u.u) v v^T; with small integers it is exact.
    u and v differ, so a transposed operand (u (v.v) u^T) fails."""
    rng = np.random.default_rng(2)
    u = rng.integers(-9, 10, size=6).astype(np.float64)
    v = rng.integers(-9, 10, size=6).astype(np.float64)
    G = oracle.gram_real(np.outer(u, v))
    assert np.array_equal(G, float(u @ u) * np.outer(v, v))


def test_orthogonal_factor_gives_identity():
    """The Q factor of a Householder QR (numpy.linalg.qr, LAPACK) is
    orthogonal: Q^T Q = I up to rounding."""
    A = np.random.default_rng(3).standard_normal((40, 40))
    Qf, _ = np.linalg.qr(A)
    assert np.max(np.abs(oracle.gram_real(Qf) - np.eye(40))) < 1e-13


@pytest.mark.parametrize("gen", [uniform_real, signed_real])
def test_exact_rational_gram_within_the_summation_bound(gen):
    """Every entry within gamma_m * sum_r |Q_ri Q_rj| of the exact Gram of the
    stored doubles, computed in rational arithmetic."""
    B, m = 3, 6
    Q = gen(B, m, 4)
    G = oracle.gram_real(Q)
    for b in range(B):
        q = [[Fraction(float(x)) for x in row] for row in Q[b]]
        for i in range(m):
            for j in range(m):
                exact = sum(q[r][i] * q[r][j] for r in range(m))
                scale = sum(abs(q[r][i] * q[r][j]) for r in range(m))
                err = abs(Fraction(float(G[b, i, j])) - exact)
                assert err <= Fraction(gamma(m, U64)) * scale


def test_batch_members_are_independent():
    """Matrix b of the batch sees only its own m x m block."""
    m = 8
    Q = np.stack([sylvester(m).astype(np.float64), 2.0 * np.eye(m), np.zeros((m, m))])
    G = oracle.gram_real(Q)
    assert np.array_equal(G[0], m * np.eye(m))
    assert np.array_equal(G[1], 4.0 * np.eye(m))
    assert np.array_equal(G[2], np.zeros((m, m)))


def test_result_is_symmetric_and_float32_is_widened_exactly():
    Q32 = uniform_real(2, 9, 5, np.float32)
    G32 = oracle.gram_real(Q32)
    G64 = oracle.gram_real(Q32.astype(np.float64))
    assert np.array_equal(G32, G64)
    assert np.array_equal(G64, np.transpose(G64, (0, 2, 1)))
