"""Failure detection without a GPU fault: the library's bounded device waits
(the persistent kernel's grid barrier, the mbarrier waits of the tensor-core
and bulk-copy pipelines) driven to their limit on targets that can never be
met, and simulated out-of-memory in the allocating calls.  Every case ends
with the context still usable: a short GA run afterwards matches the oracle."""
import time

import numpy as np
import pytest
import torch

import oracle
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def _ga_still_matches_oracle(h, m=12, N=64, gens=8):
    pop = h.Population(m, N, seed=3, storage=h.STORE_BITS, traj_cap=gens)
    pop.init_population()
    pop.fitness()
    pop.step(gens)
    pop.sync()
    got, F = pop.as_int8(), pop.fitness_host()
    pop.close()
    ref = oracle.init_population(m, 4 * N, 3)
    RF = oracle.fitness(ref, oracle.FIT_SQ)
    oracle.run(ref, RF, N, 1, 1, oracle.FIT_SQ, 3, 0, 0, gens)
    assert np.array_equal(got, ref) and np.array_equal(F, RF)


@pytest.mark.parametrize("which", [0, 1], ids=["grid_barrier", "mbarrier"])
def test_bounded_wait_runs_out_and_reports_timeout(which):
    h = need_gpu()
    t0 = time.perf_counter()
    st, word = h.debug_wait_timeout(which, 1000)   # 1 ms budget
    dt = time.perf_counter() - t0
    assert st == h.GA_ETIMEOUT
    assert word & 1                                 # ERR_TIMEOUT
    assert "budget" in h.last_error()
    assert dt < 5.0                                 # gave up after its budget, no hang
    _ga_still_matches_oracle(h)


def test_wait_timeout_rejects_bad_arguments():
    h = need_gpu()
    assert h.debug_wait_timeout(2, 1000)[0] == h.GA_EINVAL
    assert h.debug_wait_timeout(0, 0)[0] == h.GA_EINVAL
    assert h.debug_wait_timeout(1, 2_000_000)[0] == h.GA_EINVAL


def test_out_of_memory_in_create_leaves_nothing_behind():
    h = need_gpu()
    torch.cuda.synchronize()
    h.debug_fail_allocations(1)
    try:
        with pytest.raises(h.GAError) as ei:
            h.Population(20, 1000, seed=1, storage=h.STORE_BITS)
        assert ei.value.status == h.GA_ENOMEM
    finally:
        h.debug_fail_allocations(0)
    _ga_still_matches_oracle(h)


def test_out_of_memory_in_incremental_mode_keeps_the_context():
    h = need_gpu()
    m, N, gens = 40, 64, 6
    pop = h.Population(m, N, seed=2, storage=h.STORE_BITS, traj_cap=gens)
    pop.init_population()
    pop.fitness()
    h.debug_fail_allocations(1)
    try:
        with pytest.raises(h.GAError) as ei:
            pop.set_incremental(True)
        assert ei.value.status == h.GA_ENOMEM
    finally:
        h.debug_fail_allocations(0)
    pop.step(gens)          # full recomputation, as before the failed call
    pop.sync()
    ref = oracle.init_population(m, 4 * N, 2)
    RF = oracle.fitness(ref, oracle.FIT_SQ)
    oracle.run(ref, RF, N, 1, 1, oracle.FIT_SQ, 2, 0, 0, gens)
    assert np.array_equal(pop.as_int8(), ref) and np.array_equal(pop.fitness_host(), RF)
    pop.close()
