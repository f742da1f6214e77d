"""CPU oracle of the genetic algorithm's population step (arXiv 2208.14961).

TEST INFRASTRUCTURE ONLY.  The package under ``paper_2208_14961_gb300`` never
imports this module; only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` do.  The arithmetic lives in plain C
(``hadga_oracle.c``), compiled with gcc into ``oracle/_build``; this file only
marshals numpy arrays through ctypes.

Every function cites the passage of the paper it follows in the C source.
Populations are int8 arrays of shape [P, m, m] (row i, column j); fitness is
uint64 of shape [P].
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hadga_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libhadga_oracle.so")
_lock = threading.Lock()
_lib = None

FIT_SQ, FIT_ABS, FIT_NNZ = 0, 1, 2
OP_INIT, OP_SELECT, OP_CROSS, OP_MUTATE, OP_CONFIG, OP_PSELECT = 0, 1, 2, 3, 4, 5
SEL_TRUNCATION, SEL_PROBABILISTIC = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP over independent slots)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        u32, i32, i64, u64 = ctypes.c_uint32, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
        vp = ctypes.c_void_p
        sig = {
            "orc_philox4x32_10": (None, [vp, vp, vp]),
            "orc_uniform": (u32, [u32, u32, u32]),
            "orc_stream_words": (None, [u32, u32, u32, u32, u32, u32, i32, vp]),
            "orc_init_population": (None, [vp, i32, i64, u32, u32]),
            "orc_init_slots": (None, [vp, i32, vp, i64, u32, u32]),
            "orc_gram": (None, [vp, i32, vp]),
            "orc_fitness": (None, [vp, i32, i64, i64, i32, vp]),
            "orc_crossover_pair": (None, [vp, vp, vp, vp, i32, i32]),
            "orc_cut_point": (i32, [i32, u32, u32, u32, u32]),
            "orc_crossover": (None, [vp, i32, i64, u32, u32, u32]),
            "orc_mutate_explicit": (i32, [vp, i32, i32, i32, vp, vp, vp]),
            "orc_mutation_draws": (None, [i32, i32, i32, u32, u32, u32, u32, vp, vp, vp]),
            "orc_mutate": (None, [vp, i32, i64, i32, i32, u32, u32, u32, i32]),
            "orc_select_key": (u32, [u32, u32, u32, u32]),
            "orc_perm": (None, [u32, u32, u32, u32, vp]),
            "orc_survivors": (None, [vp, i64, vp]),
            "orc_select": (None, [vp, vp, i32, i64, u32, u32, u32]),
            "orc_best": (None, [vp, i64, vp, vp]),
            "orc_psel_weight": (u64, [u64]),
            "orc_psel_pick": (i64, [vp, i64, u32, u32, u32, u32]),
            "orc_select_prob": (None, [vp, vp, i32, i64, u32, u32, u32]),
            "orc_run": (i32, [vp, vp, i32, i64, i32, i32, i32, u32, u32, u32, i32, i32, vp, vp, i32, i32]),
            "orc_mixed_N": (i64, [u32, u32]),
            "orc_gram_real": (None, [vp, i32, i64, vp]),
            "orc_num_threads": (i32, []),
            "orc_set_num_threads": (None, [i32]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------------------
# RNG
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def uniform(w: int, lo: int, hi: int) -> int:
    return int(_load().orc_uniform(w, lo, hi))


def stream_words(seed, pop_id, op, gen, index, sub, count) -> np.ndarray:
    out = np.zeros(count, dtype=np.uint32)
    _load().orc_stream_words(seed, pop_id, op, gen, index, sub, count, _ptr(out))
    return out


def select_key(seed: int, pop_id: int, gen: int, d: int) -> int:
    return int(_load().orc_select_key(seed, pop_id, gen, d))


def perm(n: int, seed: int, pop_id: int, gen: int) -> np.ndarray:
    """pi of generation `gen`: parent slot p receives survivor number pi[p]."""
    out = np.zeros(max(n, 1), dtype=np.uint32)
    _load().orc_perm(n, seed, pop_id, gen, _ptr(out))
    return out[:n]


def mixed_N(seed: int, idx: int) -> int:
    return int(_load().orc_mixed_N(seed, idx))


# --------------------------------------------------------------------------
# Operators
# --------------------------------------------------------------------------
def init_population(m: int, P: int, seed: int, pop_id: int = 0) -> np.ndarray:
    pop = np.zeros((P, m, m), dtype=np.int8)
    _load().orc_init_population(_ptr(pop), m, P, seed, pop_id)
    return pop


def init_slots(m: int, slots, seed: int, pop_id: int = 0) -> np.ndarray:
    """The initial matrices of the listed slots of a population (int8
    [len(slots), m, m]), each as init_population would build it."""
    sl = np.ascontiguousarray(np.asarray(slots, dtype=np.int64))
    out = np.zeros((len(sl), m, m), dtype=np.int8)
    _load().orc_init_slots(_ptr(out), m, _ptr(sl), len(sl), seed, pop_id)
    return out


def gram(Q: np.ndarray) -> np.ndarray:
    Q = np.ascontiguousarray(Q, dtype=np.int8)
    m = Q.shape[0]
    G = np.zeros((m, m), dtype=np.int32)
    _load().orc_gram(_ptr(Q), m, _ptr(G))
    return G


def fitness(pop: np.ndarray, kind: int = FIT_SQ, first: int = 0, count: int | None = None,
            out: np.ndarray | None = None) -> np.ndarray:
    pop = np.ascontiguousarray(pop, dtype=np.int8)
    P, m = pop.shape[0], pop.shape[1]
    if count is None:
        count = P - first
    F = out if out is not None else np.zeros(P, dtype=np.uint64)
    _load().orc_fitness(_ptr(pop), m, first, count, kind, _ptr(F))
    return F


def crossover_pair(P1, P2, c):
    P1 = np.ascontiguousarray(P1, dtype=np.int8)
    P2 = np.ascontiguousarray(P2, dtype=np.int8)
    m = P1.shape[0]
    O1 = np.zeros_like(P1)
    O2 = np.zeros_like(P1)
    _load().orc_crossover_pair(_ptr(P1), _ptr(P2), _ptr(O1), _ptr(O2), m, c)
    return O1, O2


def cut_point(m, seed, pop_id, gen, k) -> int:
    return int(_load().orc_cut_point(m, seed, pop_id, gen, k))


def crossover(pop: np.ndarray, N: int, seed: int, pop_id: int, gen: int) -> None:
    _load().orc_crossover(_ptr(pop), pop.shape[1], N, seed, pop_id, gen)


def mutate_explicit(Q: np.ndarray, cols, rows1, rows2) -> int:
    """Mutates Q in place; returns the number of successful pair flips."""
    assert Q.dtype == np.int8 and Q.flags["C_CONTIGUOUS"]
    c = np.ascontiguousarray(np.asarray(cols, dtype=np.int32))
    r1 = np.ascontiguousarray(np.asarray(rows1, dtype=np.int32))
    r2 = np.ascontiguousarray(np.asarray(rows2, dtype=np.int32))
    return int(_load().orc_mutate_explicit(_ptr(Q), Q.shape[0], len(c), len(r1), _ptr(c), _ptr(r1), _ptr(r2)))


def mutation_draws(m, NC, NR, seed, pop_id, gen, o):
    c = np.zeros(NC, dtype=np.int32)
    r1 = np.zeros(NR, dtype=np.int32)
    r2 = np.zeros(NR, dtype=np.int32)
    _load().orc_mutation_draws(m, NC, NR, seed, pop_id, gen, o, _ptr(c), _ptr(r1), _ptr(r2))
    return c, r1, r2


def mutate(pop: np.ndarray, N: int, NC: int, NR: int, seed: int, pop_id: int, gen: int, shared: int = 0) -> None:
    """Mutation of the 2N offspring; shared = 1 is the paper's method 1 (one
    draw for the whole generation)."""
    _load().orc_mutate(_ptr(pop), pop.shape[1], N, NC, NR, seed, pop_id, gen, int(shared))


def survivors(F: np.ndarray, N: int) -> np.ndarray:
    F = np.ascontiguousarray(F, dtype=np.uint64)
    out = np.zeros(2 * N, dtype=np.int64)
    _load().orc_survivors(_ptr(F), N, _ptr(out))
    return out


def select(pop: np.ndarray, F: np.ndarray, N: int, seed: int, pop_id: int, gen: int) -> None:
    assert F.dtype == np.uint64
    _load().orc_select(_ptr(pop), _ptr(F), pop.shape[1], N, seed, pop_id, gen)


def psel_weight(f: int) -> int:
    """Weight of fitness f in the probabilistic selection: floor(2^32 / (f + 1))."""
    return int(_load().orc_psel_weight(f))


def psel_pick(F: np.ndarray, seed: int, pop_id: int, gen: int, p: int) -> int:
    """The individual the probabilistic selection of generation `gen` draws
    for parent slot p, given the fitness F of the whole population."""
    F = np.ascontiguousarray(F, dtype=np.uint64)
    C = np.cumsum(np.array([psel_weight(int(f)) for f in F], dtype=np.uint64)).astype(np.uint64)
    return int(_load().orc_psel_pick(_ptr(C), len(F), seed, pop_id, gen, p))


def select_prob(pop: np.ndarray, F: np.ndarray, N: int, seed: int, pop_id: int, gen: int) -> None:
    """Probabilistic selection of generation `gen` (weights inverse to F), in place."""
    assert F.dtype == np.uint64
    _load().orc_select_prob(_ptr(pop), _ptr(F), pop.shape[1], N, seed, pop_id, gen)


def best(F: np.ndarray):
    F = np.ascontiguousarray(F, dtype=np.uint64)
    s = ctypes.c_int64()
    f = ctypes.c_uint64()
    _load().orc_best(_ptr(F), F.shape[0], ctypes.byref(s), ctypes.byref(f))
    return int(s.value), int(f.value)


def run(pop: np.ndarray, F: np.ndarray, N: int, NC: int, NR: int, kind: int, seed: int,
        pop_id: int, gen0: int, generations: int, stop_at_zero: bool = False, shared_mutation: int = 0,
        selection: int = SEL_TRUNCATION):
    """Runs `generations` generations in place; returns (n_done, traj_fit, traj_slot).
    shared_mutation = 1 selects the paper's mutation method 1; selection = 1
    the probabilistic selection."""
    assert pop.dtype == np.int8 and F.dtype == np.uint64
    tf = np.zeros(max(generations, 1), dtype=np.uint64)
    ts = np.zeros(max(generations, 1), dtype=np.int64)
    n = _load().orc_run(_ptr(pop), _ptr(F), pop.shape[1], N, NC, NR, kind, seed, pop_id, gen0,
                        generations, int(stop_at_zero), _ptr(tf), _ptr(ts), int(shared_mutation), int(selection))
    return int(n), tf[:n], ts[:n]


def gram_real(Q: np.ndarray) -> np.ndarray:
    """Batched real Gram Q_b^T Q_b of a [B, m, m] (or [m, m]) array in float64
    (Sec. 2, Table 1).  float32 input is widened exactly before the loop."""
    Q = np.asarray(Q)
    single = Q.ndim == 2
    Q = np.ascontiguousarray(Q.reshape((1,) + Q.shape) if single else Q, dtype=np.float64)
    B, m = Q.shape[0], Q.shape[1]
    assert Q.shape == (B, m, m)
    G = np.zeros((B, m, m), dtype=np.float64)
    _load().orc_gram_real(_ptr(Q), m, B, _ptr(G))
    return G[0] if single else G


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_num_threads(n: int) -> None:
    _load().orc_set_num_threads(n)
