"""Helpers of the GPU parity tests (no method arithmetic here)."""
import numpy as np
import pytest
import torch


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_14961_gb300.build import build
    build()
    from paper_2208_14961_gb300 import hadga
    hadga.load()
    return hadga


def to_device_int8(pop_np):
    return torch.as_tensor(np.ascontiguousarray(pop_np)).cuda()


def fit_u64(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().view(np.uint32).astype(np.uint64)
