"""The C-ABI library loads and exports what include/hadga.h declares; host-side
argument checks answer without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hadga.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ga_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2208_14961_gb300.build import build
    build()
    from paper_2208_14961_gb300 import hadga
    return hadga.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 25
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    from paper_2208_14961_gb300 import hadga
    assert sorted(hadga.SIGNATURES) == _declared()


def test_config_struct_layout():
    from paper_2208_14961_gb300 import hadga
    assert ctypes.sizeof(hadga.ga_config) == 56
    assert hadga.ga_config.N.offset == 8
    assert hadga.ga_config.selection.offset == 48


def test_version_and_storage_bytes(lib):
    from paper_2208_14961_gb300 import hadga
    assert lib.ga_version() >= 10000
    assert hadga.storage_bytes(hadga.STORE_INT8, 20) == 400
    assert hadga.storage_bytes(hadga.STORE_BITS, 20) == 80
    assert hadga.storage_bytes(hadga.STORE_BITS, 100) == 100 * 4 * 4
    assert hadga.storage_bytes(hadga.STORE_E4M3, 32) == 1024
    assert hadga.storage_bytes(hadga.STORE_BF16, 32) == 2048
    assert hadga.storage_bytes(hadga.STORE_INT8, 18) == 0      # not a multiple of 4
    assert hadga.storage_bytes(hadga.STORE_INT8, 260) == 0     # beyond the largest order


@pytest.mark.parametrize("field,value", [("m", 18), ("m", 0), ("m", 260), ("N", 0), ("NC", 0), ("NR", 65),
                                         ("fitness", 3), ("storage", 2), ("traj_cap", 0), ("mutation", 2), ("mutation", -1),
                                         ("path", 3), ("selection", 2), ("selection", -1)])
def test_create_rejects_bad_config_without_gpu(lib, field, value):
    from paper_2208_14961_gb300 import hadga
    cfg = hadga.ga_config(m=20, NC=1, N=10, seed=0, pop_id=0, NR=1, fitness=0, storage=1, path=0,
                          traj_cap=8, mutation=0)
    setattr(cfg, field, value)
    ctx = ctypes.c_void_p()
    buf = ctypes.c_void_p(0x1000)  # never dereferenced: validation fails first
    st = lib.ga_create(ctypes.byref(cfg), buf, buf, None, ctypes.byref(ctx))
    assert st == hadga.GA_EINVAL
    assert not ctx.value
    assert hadga.last_error()


def test_null_arguments(lib):
    from paper_2208_14961_gb300 import hadga
    assert lib.ga_create(None, None, None, None, None) == hadga.GA_EINVAL
    assert lib.ga_select(None) == hadga.GA_EINVAL
    assert lib.ga_destroy(None) == hadga.GA_OK
    assert lib.ga_step_multi(None, 0, 1) == hadga.GA_EINVAL
    assert lib.ga_fitness_batch(None, 0, 20, 10, 0, 0, None, None) == hadga.GA_EINVAL
    assert lib.ga_convert(None, 0, None, 1, 20, 10, None) == hadga.GA_EINVAL
    assert "NULL" in hadga.last_error() or hadga.last_error()


def test_misaligned_buffers_rejected(lib):
    from paper_2208_14961_gb300 import hadga
    cfg = hadga.ga_config(m=20, NC=1, N=10, seed=0, pop_id=0, NR=1, fitness=0, storage=1, path=0,
                          traj_cap=8, mutation=0)
    ctx = ctypes.c_void_p()
    st = lib.ga_create(ctypes.byref(cfg), ctypes.c_void_p(0x1004), ctypes.c_void_p(0x2000), None, ctypes.byref(ctx))
    assert st == hadga.GA_EINVAL and "aligned" in hadga.last_error()


def test_package_has_no_cpu_fallback():
    """The product package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2208_14961_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f


@pytest.mark.parametrize("typ,m,B,same", [(2, 8, 1, False), (-1, 8, 1, False), (1, 0, 1, False), (1, 257, 1, False),
                                          (0, 8, -1, False), (1, 8, 1, True)])
def test_gram_real_rejects_bad_arguments_without_gpu(lib, typ, m, B, same):
    from paper_2208_14961_gb300 import hadga
    q = ctypes.c_void_p(0x10000)
    g = q if same else ctypes.c_void_p(0x90000000)
    assert lib.ga_gram_real_batch(q, g, typ, m, B, None) == hadga.GA_EINVAL
    assert hadga.last_error()


def test_gram_real_rejects_misaligned_buffers(lib):
    from paper_2208_14961_gb300 import hadga
    st = lib.ga_gram_real_batch(ctypes.c_void_p(0x10008), ctypes.c_void_p(0x90000000), 1, 8, 1, None)
    assert st == hadga.GA_EINVAL and "bad buffers" in hadga.last_error()


def test_gram_real_empty_batch_accepts_null_buffers(lib):
    from paper_2208_14961_gb300 import hadga
    assert lib.ga_gram_real_batch(None, None, 1, 8, 0, None) == hadga.GA_OK
    assert lib.ga_gram_real_batch(None, None, 0, 256, 0, None) == hadga.GA_OK


def test_binding_constants_match_the_header():
    """Every enum value include/hadga.h declares has the same value in the
    binding (GA_FIT_SQ -> FIT_SQ, GA_PATH_POPC -> PATH_POPC, ...)."""
    from paper_2208_14961_gb300 import hadga
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    consts = dict((n, int(v)) for n, v in re.findall(r"\b(GA_[A-Z0-9_]+)\s*=\s*([0-9]+)", src))
    assert len(consts) >= 22
    for name, value in consts.items():
        short = name if hasattr(hadga, name) else name[3:]
        assert getattr(hadga, short) == value, name


# ga_select_static: every output must stay clear of every input and of the
# other output (the gather writes parent_fit_out[p] while fit_in[src] is still
# read).  Buffers are fake addresses: validation answers before any device call.
_N_SS, _M_SS = 8, 20          # BITS storage: 80 bytes per matrix
_POP, _FIT = 0x100000, 0x200000
_PAR, _PFIT = 0x300000, 0x400000


@pytest.mark.parametrize("par,pfit,what", [
    (_POP + 16, _PFIT, "parents_out must not overlap pop_in"),
    (_PAR, _FIT, "parent_fit_out must not overlap fit_in"),
    (_FIT - 16, _PFIT, "parents_out must not overlap fit_in"),
    (_PAR, _POP + 4 * _N_SS * 80 - 16, "parent_fit_out must not overlap pop_in"),
    (_PAR, _PAR + 2 * _N_SS * 80 - 16, "parents_out must not overlap parent_fit_out"),
])
def test_select_static_rejects_every_overlap(lib, par, pfit, what):
    from paper_2208_14961_gb300 import hadga
    st = lib.ga_select_static(ctypes.c_void_p(_POP), ctypes.c_void_p(_FIT), ctypes.c_void_p(par),
                              ctypes.c_void_p(pfit), hadga.STORE_BITS, _M_SS, _N_SS, 0, 0, 1, None)
    assert st == hadga.GA_EINVAL
    assert what in hadga.last_error()


def test_select_static_error_rejects_null(lib):
    """The error-word accessor validates its output pointer before any device call."""
    from paper_2208_14961_gb300 import hadga
    assert lib.ga_select_static_error(None, None) == hadga.GA_EINVAL
    assert "NULL err_out" in hadga.last_error()


def test_out_of_memory_hook_in_create_without_gpu(lib):
    """The allocation-failure hook makes ga_create fail with GA_ENOMEM before
    the allocator is called, and return no context (host side only: the
    buffers are fake and never touched)."""
    from paper_2208_14961_gb300 import hadga
    cfg = hadga.ga_config(m=20, NC=1, N=10, seed=0, pop_id=0, NR=1, fitness=0, storage=1, path=0,
                          traj_cap=8, mutation=0)
    ctx = ctypes.c_void_p()
    assert lib.ga_debug_fail_allocations(-1) == hadga.GA_EINVAL
    assert lib.ga_debug_fail_allocations(1) == hadga.GA_OK
    try:
        st = lib.ga_create(ctypes.byref(cfg), ctypes.c_void_p(0x100000), ctypes.c_void_p(0x200000), None,
                           ctypes.byref(ctx))
    finally:
        lib.ga_debug_fail_allocations(0)
    assert st == hadga.GA_ENOMEM
    assert not ctx.value
    assert "allocation" in hadga.last_error()


def test_shape_and_auto_path_setters_validate_without_gpu(lib):
    from paper_2208_14961_gb300 import hadga
    assert lib.ga_set_fused_shape(None, 2, 0) == hadga.GA_EINVAL
    # a path that does not read the storage is refused; a valid one is kept and cleared
    assert lib.ga_set_auto_path(hadga.STORE_BITS, 20, hadga.FIT_SQ, hadga.PATH_IMMA) == hadga.GA_EINVAL
    assert lib.ga_set_auto_path(hadga.STORE_BITS, 20, hadga.FIT_SQ, 9) == hadga.GA_EINVAL
    assert lib.ga_set_auto_path(hadga.STORE_BITS, 18, hadga.FIT_SQ, hadga.PATH_POPC) == hadga.GA_EINVAL
    assert lib.ga_set_auto_path(hadga.STORE_BITS, 20, hadga.FIT_SQ, hadga.PATH_POPC) == hadga.GA_OK
    assert lib.ga_set_auto_path(hadga.STORE_BITS, 20, hadga.FIT_SQ, hadga.PATH_AUTO) == hadga.GA_OK
