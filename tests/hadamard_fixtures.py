"""Known Hadamard matrices and the paper's worked examples, as test fixtures.

Sylvester's doubling and Paley's first construction (quadratic residues
modulo a prime q = 3 mod 4) are textbook constructions, written here with
numpy only; every matrix is normalised so that its first column is all +1.
The golden files under tests/golden/ hold the paper's printed examples.
"""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def normalise(H: np.ndarray) -> np.ndarray:
    """Negate rows so that column 0 is all +1 (keeps H Hadamard)."""
    return (H * H[:, :1]).astype(np.int8)


def sylvester(m: int) -> np.ndarray:
    H = np.ones((1, 1), dtype=np.int64)
    while H.shape[0] < m:
        H = np.block([[H, H], [H, -H]])
    assert H.shape[0] == m, "m must be a power of two"
    return normalise(H)


def paley1(q: int) -> np.ndarray:
    """Order q + 1 Hadamard matrix for a prime q = 3 (mod 4)."""
    assert q % 4 == 3 and all(q % d for d in range(2, int(q ** 0.5) + 1))
    residues = {(x * x) % q for x in range(1, q)}
    chi = np.array([0] + [1 if a in residues else -1 for a in range(1, q)], dtype=np.int64)
    J = np.array([[chi[(j - i) % q] for j in range(q)] for i in range(q)], dtype=np.int64)
    S = np.zeros((q + 1, q + 1), dtype=np.int64)
    S[0, 1:] = 1
    S[1:, 0] = -1
    S[1:, 1:] = J
    H = S + np.eye(q + 1, dtype=np.int64)
    return normalise(H)


def _rows(lines):
    return np.array([[1 if ch == "+" else -1 for ch in ln.replace(" ", "")] for ln in lines], dtype=np.int8)


def _content(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return [ln.rstrip("\n") for ln in fh if ln.strip() and not ln.startswith("#")]


def philox_kat():
    out = []
    for ln in _content("philox4x32_10_kat.txt"):
        v = [int(x, 16) for x in ln.split()]
        out.append((v[0:4], v[4:6], v[6:10]))
    return out


def crossover_fig2():
    lines = _content("crossover_fig2.txt")
    cut = int(lines[0].split()[1])
    mats = {}
    i = 1
    while i < len(lines):
        name = lines[i].strip()
        mats[name] = _rows(lines[i + 1:i + 5])
        i += 5
    return cut, mats


def mutation_fig3():
    lines = _content("mutation_fig3.txt")
    parts, cur, i = {}, None, 0
    while i < len(lines):
        tok = lines[i].split()
        if tok[0] == "part":
            cur = {}
            parts[tok[1]] = cur
        elif tok[0] == "cols":
            cur["cols"] = [int(x) for x in tok[1:]]
        elif tok[0] in ("pairs", "printed_pairs"):
            cur[tok[0]] = [tuple(int(y) for y in x.split(",")) for x in tok[1:]]
        elif tok[0] in ("success", "fail"):
            cur[tok[0]] = {tuple(int(y) for y in x.split(",")) for x in tok[1:]}
        elif tok[0] == "matrix":
            cur["matrix"] = _rows(lines[i + 1:i + 9])
            i += 8
        i += 1
    return parts
