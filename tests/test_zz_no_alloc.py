"""ga_select_static: the selection step for callers that cannot allocate
device memory while it runs (its scratch is a fixed array inside the
library).  Checked against the context-based ga_select and the oracle's
selection, bit for bit, on two calls in a row, with the step's device error
word (its survivor-count and mask consistency checks) read back as zero
after each call.  Named to be collected last."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def _as_int8(h, t, storage, m, P):
    if storage == h.STORE_INT8:
        return t.cpu().numpy().copy()
    out = h.empty_population(h.STORE_INT8, m, P)
    h.ga_convert(t, storage, out, h.STORE_INT8, m, P)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("storage,m,N", [(1, 20, 2500), (0, 12, 8192)])
def test_select_static_matches_ga_select(storage, m, N):
    h = need_gpu()
    seed, pop_id = 5, 1
    ref = h.Population(m, N, seed=seed, pop_id=pop_id, storage=storage)
    ref.init_population()
    ref.fitness()
    torch.cuda.synchronize()
    pop_in = ref.pop.clone()
    fit_in = ref.fit.clone()
    shape, dt = h.storage_shape(storage, m, 2 * N)
    for call in range(2):       # two calls in a row on the shared array
        gen = call + 1
        parents = torch.empty(shape, dtype=dt, device="cuda")
        pfit = torch.empty(2 * N, dtype=torch.int32, device="cuda")
        h.ga_select_static(pop_in, fit_in, parents, pfit, storage, m, N, seed, pop_id, gen,
                           stream=torch.cuda.current_stream())
        assert h.ga_select_static_error(stream=torch.cuda.current_stream()) == 0
        ref.select()            # the existing entry point, generation `gen`
        torch.cuda.synchronize()
        assert ref.generation() == gen
        assert torch.equal(parents, ref.pop[:2 * N])
        assert torch.equal(pfit, ref.fit[:2 * N])
        # and the oracle's selection of the same generation (Sec. 3.3)
        host_in = _as_int8(h, pop_in, storage, m, 4 * N)
        F = fit_in.cpu().numpy().view(np.uint32).astype(np.uint64)
        oracle.select(host_in, F, N, seed, pop_id, gen)
        assert np.array_equal(_as_int8(h, parents, storage, m, 2 * N), host_in[:2 * N])
        assert np.array_equal(pfit.cpu().numpy().view(np.uint32).astype(np.uint64), F[:2 * N])
        # next call: the population after this selection
        pop_in = ref.pop.clone()
        fit_in = ref.fit.clone()
    ref.close()


def test_select_static_rejects_too_large_population():
    h = need_gpu()
    N = 8193
    pop = torch.empty((4 * N, 4, 1), dtype=torch.int32, device="cuda")
    fit = torch.zeros(4 * N, dtype=torch.int32, device="cuda")
    out = torch.empty((2 * N, 4, 1), dtype=torch.int32, device="cuda")
    of = torch.empty(2 * N, dtype=torch.int32, device="cuda")
    with pytest.raises(h.GAError) as ei:
        h.ga_select_static(pop, fit, out, of, 1, 4, N, 0, 0, 1)
    assert ei.value.status == h.GA_EINVAL and "8192" in str(ei.value)
