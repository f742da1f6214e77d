"""Seeded synthetic inputs shared by the oracle tests and the GPU parity tests.

This module holds no arithmetic of the method (no Gram, no fitness, no
operator): it only draws populations with numpy's own seeded generator.
"""
import numpy as np


def random_pm1(P: int, m: int, seed: int) -> np.ndarray:
    """Unstructured +-1 matrices (columns not balanced), int8 [P, m, m]."""
    rng = np.random.default_rng(seed)
    return np.where(rng.random((P, m, m)) < 0.5, -1, 1).astype(np.int8)


def balanced_pm1(P: int, m: int, seed: int) -> np.ndarray:
    """Column 0 all +1, every other column a random arrangement of m/2 (+1)
    and m/2 (-1), drawn with numpy (independent of the method's RNG)."""
    rng = np.random.default_rng(seed)
    base = np.concatenate([-np.ones(m // 2, np.int8), np.ones(m - m // 2, np.int8)])
    pop = np.ones((P, m, m), dtype=np.int8)
    keys = rng.random((P, m - 1, m))
    order = np.argsort(keys, axis=2)              # a random permutation per column
    cols = base[order]                            # [P, m-1, m]
    pop[:, :, 1:] = np.transpose(cols, (0, 2, 1))
    return pop
