"""Throughput microbenchmarks used as the compute roofs of the kernels
(popcount, dp4a, IMAD, warp-level s8 and e4m3 MMA, FP64 and FP32 FMA), the
L2 read rate and the grid-barrier latency; built into _build/libpeaks.so."""
import ctypes
import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = os.path.join(os.path.dirname(_HERE), "_build", "libpeaks.so")

KINDS = {"popc": 0, "popc_chain": 1, "dp4a": 2, "imma_s8": 3, "imad": 4, "mma_e4m3": 5, "l2_read_bytes": 6,
         "grid_barriers": 7, "dfma": 8, "ffma": 9}


def build():
    src = os.path.join(_HERE, "peaks.cu")
    if os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(src):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
                    "-shared", "-I", os.path.join(os.path.dirname(_HERE), "csrc"), "-o", _LIB, src], check=True)
    return _LIB


def rate(kind: str, iters: int = 4096) -> float:
    lib = ctypes.CDLL(build())
    lib.peak_rate.restype = ctypes.c_double
    lib.peak_rate.argtypes = [ctypes.c_int, ctypes.c_int]
    return float(lib.peak_rate(KINDS[kind], iters))
