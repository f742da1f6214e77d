"""Thin ctypes binding of libhadga (include/hadga.h).

Argument marshalling only: every step of the genetic algorithm runs in the
CUDA kernels of ``libhadga.so``.  Device buffers are torch tensors (device
memory and streams are the only things torch provides here).  There is no
CPU fallback: importing this module without a built library, or calling it
without a CUDA device, raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhadga.so")

GA_OK, GA_EINVAL, GA_ENOMEM, GA_ECUDA, GA_ETIMEOUT, GA_EUNSUPPORTED = range(6)
FIT_SQ, FIT_ABS, FIT_NNZ = 0, 1, 2
STORE_INT8, STORE_BITS, STORE_E4M3, STORE_BF16 = 0, 1, 2, 3
PATH_AUTO, PATH_INT32, PATH_IMMA, PATH_FP8, PATH_BF16, PATH_POPC, PATH_FP8_WARP = range(7)
GA_REAL_F32, GA_REAL_F64 = 0, 1
SEL_TRUNCATION, SEL_PROBABILISTIC = 0, 1

_STATUS_NAMES = {0: "GA_OK", 1: "GA_EINVAL", 2: "GA_ENOMEM", 3: "GA_ECUDA", 4: "GA_ETIMEOUT",
                 5: "GA_EUNSUPPORTED"}


class GAError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class ga_config(ctypes.Structure):
    _fields_ = [
        ("m", ctypes.c_int32),
        ("NC", ctypes.c_int32),
        ("N", ctypes.c_int64),
        ("seed", ctypes.c_uint32),
        ("pop_id", ctypes.c_uint32),
        ("NR", ctypes.c_int32),
        ("fitness", ctypes.c_int32),
        ("storage", ctypes.c_int32),
        ("path", ctypes.c_int32),
        ("traj_cap", ctypes.c_int32),
        ("mutation", ctypes.c_int32),
        ("selection", ctypes.c_int32),
    ]


# name -> (restype, argtypes); the full set of symbols include/hadga.h declares
_vp, _i32, _i64, _u32, _sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_size_t
SIGNATURES = {
    "ga_version": (_i32, []),
    "ga_storage_bytes": (_sz, [_i32, _i32]),
    "ga_create": (_i32, [ctypes.POINTER(ga_config), _vp, _vp, _vp, ctypes.POINTER(_vp)]),
    "ga_destroy": (_i32, [_vp]),
    "ga_init_population": (_i32, [_vp]),
    "ga_fitness": (_i32, [_vp, _i64, _i64]),
    "ga_select": (_i32, [_vp]),
    "ga_crossover": (_i32, [_vp]),
    "ga_mutate": (_i32, [_vp]),
    "ga_record_best": (_i32, [_vp]),
    "ga_step_plain": (_i32, [_vp, _i32]),
    "ga_step": (_i32, [_vp, _i32, _i32, ctypes.POINTER(_i32)]),
    "ga_step_multi": (_i32, [ctypes.POINTER(_vp), _i32, _i32]),
    "ga_step_is_fused": (_i32, [_vp]),
    "ga_set_strict": (_i32, [_vp, _i32]),
    "ga_step_multi_graph": (_i32, [ctypes.POINTER(_vp), _i32, _i32, _i32]),
    "ga_set_fused_grid": (_i32, [_vp, _i32]),
    "ga_set_fused_shape": (_i32, [_vp, _i32, _i32]),
    "ga_set_auto_path": (_i32, [_i32, _i32, _i32, _i32]),
    "ga_set_incremental": (_i32, [_vp, _i32]),
    "ga_check_incremental": (_i32, [_vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
    "ga_get_incremental": (_i32, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_float),
                                   ctypes.POINTER(ctypes.c_float)]),
    "ga_get_gram": (_i32, [_vp, _i64, _vp]),
    "ga_best": (_i32, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_u32)]),
    "ga_trajectory": (_i32, [_vp, _vp, _vp, _i32, ctypes.POINTER(_i32)]),
    "ga_generation": (_i32, [_vp, ctypes.POINTER(_u32)]),
    "ga_set_generation": (_i32, [_vp, _u32]),
    "ga_sync": (_i32, [_vp]),
    "ga_set_slot": (_i32, [_vp, _i64, _vp]),
    "ga_get_slot": (_i32, [_vp, _i64, _vp]),
    "ga_last_error": (ctypes.c_char_p, [_vp]),
    "ga_kernel_launches": (ctypes.c_uint64, []),
    "ga_profile": (_i32, [_vp, _i32]),
    "ga_profile_read": (_i32, [_vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                                ctypes.POINTER(_i32)]),
    "ga_init_batch": (_i32, [_vp, _i32, _i32, _i64, _u32, _u32, _vp]),
    "ga_fitness_batch": (_i32, [_vp, _i32, _i32, _i64, _i32, _i32, _vp, _vp]),
    "ga_convert": (_i32, [_vp, _i32, _vp, _i32, _i32, _i64, _vp]),
    "ga_gram_real_batch": (_i32, [_vp, _vp, _i32, _i32, _i64, _vp]),
    "ga_select_static": (_i32, [_vp, _vp, _vp, _vp, _i32, _i32, _i64, _u32, _u32, _u32, _vp]),
    "ga_select_static_error": (_i32, [ctypes.POINTER(_u32), _vp]),
    "ga_debug_wait_timeout": (_i32, [_i32, _u32, ctypes.POINTER(_u32), _vp]),
    "ga_debug_fail_allocations": (_i32, [_i32]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Loads libhadga.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libhadga.so not built at {path}; run paper_2208_14961_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def last_error(ctx=None) -> str:
    msg = load().ga_last_error(ctx)
    return msg.decode() if msg else ""


def check(status: int, ctx=None) -> None:
    if status != GA_OK:
        raise GAError(status, last_error(ctx))


def _ptr(t: torch.Tensor):
    if not t.is_cuda:
        raise ValueError("libhadga works on CUDA tensors only")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def kernel_launches() -> int:
    return int(load().ga_kernel_launches())


def storage_bytes(storage: int, m: int) -> int:
    return int(load().ga_storage_bytes(storage, m))


def storage_shape(storage: int, m: int, P: int):
    """(shape, dtype) of a torch tensor holding P matrices in `storage`."""
    if storage == STORE_INT8:
        return (P, m, m), torch.int8
    if storage == STORE_BITS:
        return (P, m, (m + 31) // 32), torch.int32
    if storage == STORE_E4M3:
        return (P, m, m), torch.uint8
    if storage == STORE_BF16:
        return (P, m, m), torch.int16
    raise ValueError(storage)


def empty_population(storage: int, m: int, P: int, device="cuda") -> torch.Tensor:
    shape, dt = storage_shape(storage, m, P)
    return torch.empty(shape, dtype=dt, device=device)


# ---------------------------------------------------------------------------
# Stateless batch calls
# ---------------------------------------------------------------------------
def ga_init_batch(pop: torch.Tensor, storage: int, m: int, P: int, seed: int, pop_id: int = 0, stream=None):
    check(load().ga_init_batch(_ptr(pop), storage, m, P, seed, pop_id, _stream(stream)))


def ga_fitness_batch(pop: torch.Tensor, storage: int, m: int, P: int, kind: int, path: int,
                     fit: torch.Tensor, stream=None):
    check(load().ga_fitness_batch(_ptr(pop), storage, m, P, kind, path, _ptr(fit), _stream(stream)))


def ga_convert(src: torch.Tensor, src_storage: int, dst: torch.Tensor, dst_storage: int, m: int, P: int,
               stream=None):
    check(load().ga_convert(_ptr(src), src_storage, _ptr(dst), dst_storage, m, P, _stream(stream)))


def ga_gram_real_batch(q: torch.Tensor, g: torch.Tensor, stream=None):
    """G_b = Q_b^T Q_b for a [B, m, m] float32 or float64 tensor into g (same
    shape and dtype); the batched product of the speed comparison of Sec. 2."""
    if q.dtype not in (torch.float32, torch.float64) or g.dtype != q.dtype or g.shape != q.shape:
        raise ValueError("q and g must be float32 or float64 tensors of one shape [B, m, m]")
    if q.dim() != 3 or q.shape[1] != q.shape[2]:
        raise ValueError("q must have shape [B, m, m]")
    typ = GA_REAL_F64 if q.dtype == torch.float64 else GA_REAL_F32
    check(load().ga_gram_real_batch(_ptr(q), _ptr(g), typ, q.shape[1], q.shape[0], _stream(stream)))


def ga_select_static(pop_in: torch.Tensor, fit_in: torch.Tensor, parents_out: torch.Tensor,
                     parent_fit_out: torch.Tensor, storage: int, m: int, N: int, seed: int, pop_id: int, gen: int,
                     stream=None):
    """Selection of generation `gen` into caller buffers, with no device
    allocation (the scratch is a fixed array inside the library)."""
    check(load().ga_select_static(_ptr(pop_in), _ptr(fit_in), _ptr(parents_out), _ptr(parent_fit_out), storage, m,
                                  N, seed, pop_id, gen, _stream(stream)))


def ga_select_static_error(stream=None) -> int:
    """Error word of the last ga_select_static call ordered before `stream`
    (synchronises it): 0 when its consistency checks held."""
    w = ctypes.c_uint32(0)
    check(load().ga_select_static_error(ctypes.byref(w), _stream(stream)))
    return int(w.value)


def debug_wait_timeout(which: int, budget_us: int, stream=None):
    """Test hook: drives a bounded device wait (0 grid barrier, 1 mbarrier)
    to its limit; returns (status, device error word) without raising."""
    w = ctypes.c_uint32(0)
    st = load().ga_debug_wait_timeout(which, budget_us, ctypes.byref(w), _stream(stream))
    return int(st), int(w.value)


def debug_fail_allocations(n: int):
    """Test hook: the next n device allocations of the library fail (GA_ENOMEM)."""
    check(load().ga_debug_fail_allocations(n))


# ---------------------------------------------------------------------------
# Context
# ---------------------------------------------------------------------------
class Population:
    """A GA context over torch-owned device buffers (population + fitness)."""

    def __init__(self, m: int, N: int, seed: int = 0, pop_id: int = 0, NC: int = 1, NR: int = 1,
                 fitness: int = FIT_SQ, storage: int = STORE_BITS, path: int = PATH_AUTO,
                 traj_cap: int = 1024, device="cuda", stream=None, mutation: int = 0,
                 selection: int = SEL_TRUNCATION):
        lib = load()
        self.m, self.N, self.P = m, N, 4 * N
        self.storage = storage
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        self.pop = empty_population(storage, m, self.P, device)
        self.fit = torch.zeros(self.P, dtype=torch.int32, device=device)
        self.cfg = ga_config(m=m, NC=NC, N=N, seed=seed, pop_id=pop_id, NR=NR, fitness=fitness,
                             storage=storage, path=path, traj_cap=traj_cap, mutation=mutation,
                             selection=selection)
        ctx = ctypes.c_void_p()
        check(lib.ga_create(ctypes.byref(self.cfg), _ptr(self.pop), _ptr(self.fit),
                            ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(ctx)))
        self.ctx = ctx
        self.traj_cap = traj_cap
        self.incremental = False

    def close(self):
        if getattr(self, "ctx", None):
            load().ga_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, status):
        check(status, self.ctx)

    def init_population(self):
        self._chk(load().ga_init_population(self.ctx))

    def fitness(self, first: int = 0, count: int | None = None):
        self._chk(load().ga_fitness(self.ctx, first, self.P - first if count is None else count))

    def select(self):
        self._chk(load().ga_select(self.ctx))

    def crossover(self):
        self._chk(load().ga_crossover(self.ctx))

    def mutate(self):
        self._chk(load().ga_mutate(self.ctx))

    def record_best(self):
        self._chk(load().ga_record_best(self.ctx))

    def step_plain(self, generations: int):
        self._chk(load().ga_step_plain(self.ctx, generations))

    def step(self, generations: int, stop_at_zero: bool = False, want_done: bool = False):
        done = ctypes.c_int32(0)
        self._chk(load().ga_step(self.ctx, generations, int(stop_at_zero),
                                 ctypes.byref(done) if (want_done or stop_at_zero) else None))
        return int(done.value)

    def is_fused(self) -> bool:
        return bool(load().ga_step_is_fused(self.ctx))

    def set_strict(self, strict: bool = True):
        """ga_step raises GA_EUNSUPPORTED instead of falling back to the plain path."""
        self._chk(load().ga_set_strict(self.ctx, int(strict)))

    def profile(self, enable: bool):
        self._chk(load().ga_profile(self.ctx, int(enable)))

    def profile_read(self):
        a, b, n = ctypes.c_float(), ctypes.c_float(), ctypes.c_int32()
        self._chk(load().ga_profile_read(self.ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(n)))
        return float(a.value), float(b.value), int(n.value)

    def set_incremental(self, enable):
        """a7: keep each individual's Gram and update it by deltas in ga_step.
        enable: True / False, or "auto" to keep whichever of the two modes a
        short timed run from the current population finds faster."""
        mode = 2 if enable == "auto" else int(bool(enable))
        self._chk(load().ga_set_incremental(self.ctx, mode))
        self.incremental = self.incremental_choice()[0]

    def incremental_choice(self):
        """(incremental on, full ms/generation, incremental ms/generation) of the last AUTO choice."""
        en, a, b = ctypes.c_int32(), ctypes.c_float(), ctypes.c_float()
        self._chk(load().ga_get_incremental(self.ctx, ctypes.byref(en), ctypes.byref(a), ctypes.byref(b)))
        return bool(en.value), float(a.value), float(b.value)

    def check_incremental(self):
        """Full recomputation check: (mismatched Gram entries, mismatched fitness words)."""
        e, f = ctypes.c_uint64(), ctypes.c_uint64()
        self._chk(load().ga_check_incremental(self.ctx, ctypes.byref(e), ctypes.byref(f)))
        return int(e.value), int(f.value)

    def gram(self, slot: int):
        """Stored Gram G (m x m int32) of one slot in incremental mode."""
        import numpy as np
        g = np.zeros((self.m, self.m), dtype=np.int32)
        self._chk(load().ga_get_gram(self.ctx, slot, g.ctypes.data_as(ctypes.c_void_p)))
        return g

    def best(self):
        s, f = ctypes.c_int64(), ctypes.c_uint32()
        self._chk(load().ga_best(self.ctx, ctypes.byref(s), ctypes.byref(f)))
        return int(s.value), int(f.value)

    def trajectory(self):
        import numpy as np
        fit = np.zeros(self.traj_cap, dtype=np.uint32)
        slot = np.zeros(self.traj_cap, dtype=np.int64)
        n = ctypes.c_int32()
        self._chk(load().ga_trajectory(self.ctx, fit.ctypes.data_as(ctypes.c_void_p),
                                       slot.ctypes.data_as(ctypes.c_void_p), self.traj_cap, ctypes.byref(n)))
        return fit[:n.value], slot[:n.value]

    def generation(self) -> int:
        g = ctypes.c_uint32()
        self._chk(load().ga_generation(self.ctx, ctypes.byref(g)))
        return int(g.value)

    def set_generation(self, g: int):
        self._chk(load().ga_set_generation(self.ctx, g))

    def sync(self):
        self._chk(load().ga_sync(self.ctx))

    def set_slot(self, slot: int, matrix):
        import numpy as np
        a = np.ascontiguousarray(matrix, dtype=np.int8)
        assert a.shape == (self.m, self.m)
        self._chk(load().ga_set_slot(self.ctx, slot, a.ctypes.data_as(ctypes.c_void_p)))

    def get_slot(self, slot: int):
        import numpy as np
        a = np.zeros((self.m, self.m), dtype=np.int8)
        self._chk(load().ga_get_slot(self.ctx, slot, a.ctypes.data_as(ctypes.c_void_p)))
        return a

    def as_int8(self):
        """The whole population as a host int8 array [P, m, m] (via the GPU)."""
        if self.storage == STORE_INT8:
            return self.pop.cpu().numpy()
        out = empty_population(STORE_INT8, self.m, self.P, self.pop.device)
        ga_convert(self.pop, self.storage, out, STORE_INT8, self.m, self.P, self.stream)
        torch.cuda.synchronize()
        return out.cpu().numpy()

    def load_int8(self, host_pop):
        """Replaces the population by a host int8 array [P, m, m]."""
        t = torch.as_tensor(host_pop, dtype=torch.int8).to(self.pop.device).contiguous()
        if self.storage == STORE_INT8:
            self.pop.copy_(t)
        else:
            ga_convert(t, STORE_INT8, self.pop, self.storage, self.m, self.P, self.stream)
        torch.cuda.synchronize()
        if self.incremental:
            self.set_incremental(True)  # rebuild the Gram storage of the new population

    def fitness_host(self):
        import numpy as np
        torch.cuda.synchronize()
        return self.fit.cpu().numpy().view(np.uint32).astype(np.uint64)


def step_multi(pops, generations: int):
    arr = (ctypes.c_void_p * len(pops))(*[p.ctx for p in pops])
    check(load().ga_step_multi(arr, len(pops), generations))


def step_multi_graph(pops, generations: int, chunk: int = 50):
    arr = (ctypes.c_void_p * len(pops))(*[p.ctx for p in pops])
    check(load().ga_step_multi_graph(arr, len(pops), generations, chunk))


def set_fused_grid(pop, blocks: int):
    check(load().ga_set_fused_grid(pop.ctx, blocks))


def set_fused_shape(pop, tpp: int = 0, nch: int = 0):
    """Per-population launch shape of the persistent kernel (see ga_set_fused_shape)."""
    check(load().ga_set_fused_shape(pop.ctx, tpp, nch), pop.ctx)


def set_auto_path(storage: int, m: int, kind: int, path: int):
    """Process-wide GA_PATH_AUTO override for (storage, m, kind)."""
    check(load().ga_set_auto_path(storage, m, kind, path))
