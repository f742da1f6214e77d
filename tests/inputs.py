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


def uniform_real(B: int, m: int, seed: int, dtype=np.float64) -> np.ndarray:
    """B real m x m matrices with entries uniform on [0, 1), the input of the
    batched-Gram speed comparison (Sec. 2, Table 1: N = 10,000, m = 100)."""
    rng = np.random.default_rng(seed)
    return rng.random((B, m, m)).astype(dtype)


def signed_real(B: int, m: int, seed: int, dtype=np.float64) -> np.ndarray:
    """Entries uniform on [-1, 1) scaled by random powers of two (2^-8 .. 2^8),
    so that sums cancel and magnitudes spread."""
    rng = np.random.default_rng(seed)
    x = rng.random((B, m, m)) * 2.0 - 1.0
    return (x * np.exp2(rng.integers(-8, 9, size=(B, m, m)))).astype(dtype)
