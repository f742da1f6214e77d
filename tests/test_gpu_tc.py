"""tcgen05 (FP8 e4m3 / BF16, FP32 accumulate in TMEM) Gram + F_sq against
the oracle, bit for bit: ragged populations (partial last tile), every
supported order, and known Hadamard matrices."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import fit_u64, need_gpu, to_device_int8
from hadamard_fixtures import sylvester
from inputs import balanced_pm1, random_pm1

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m", [32, 64, 128, 256])
@pytest.mark.parametrize("storage,path", [(2, 3), (3, 4)])
def test_tc_fsq_matches_oracle(m, storage, path):
    h = need_gpu()
    P = {32: 45, 64: 23, 128: 7, 256: 5}[m]
    host = np.concatenate([random_pm1(P - 3, m, seed=m), balanced_pm1(3, m, seed=m + 1)])
    pop = h.empty_population(storage, m, P)
    h.ga_convert(to_device_int8(host), 0, pop, storage, m, P)
    fit = torch.zeros(P, dtype=torch.int32, device="cuda")
    h.ga_fitness_batch(pop, storage, m, P, h.FIT_SQ, path, fit)
    assert np.array_equal(fit_u64(fit), oracle.fitness(host, oracle.FIT_SQ))


@pytest.mark.parametrize("storage,path", [(2, 3), (3, 4)])
def test_tc_sylvester_is_optimal(storage, path):
    h = need_gpu()
    for m in (32, 64, 128, 256):
        H = sylvester(m)
        pop = h.empty_population(storage, m, 2)
        h.ga_convert(to_device_int8(np.stack([H, H])), 0, pop, storage, m, 2)
        fit = torch.full((2,), 9, dtype=torch.int32, device="cuda")
        h.ga_fitness_batch(pop, storage, m, 2, h.FIT_SQ, path, fit)
        assert fit_u64(fit).tolist() == [0, 0]


def test_tc_rejects_other_kinds_and_orders():
    h = need_gpu()
    pop = h.empty_population(2, 32, 4)
    fit = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(h.GAError) as e:
        h.ga_fitness_batch(pop, 2, 32, 4, h.FIT_NNZ, 3, fit)
    assert e.value.status == h.GA_EUNSUPPORTED
    pop = h.empty_population(2, 20, 4)
    with pytest.raises(h.GAError) as e:
        h.ga_fitness_batch(pop, 2, 20, 4, h.FIT_SQ, 3, fit)
    assert e.value.status == h.GA_EUNSUPPORTED
