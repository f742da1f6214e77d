"""GPU parity of whole generations (plain operators and the fused
persistent kernel) against the oracle's generation loop."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def _run_gpu(h, m, N, seed, gens, storage, mode, NC=1, NR=1, kind=0, pop_id=0):
    pop = h.Population(m, N, seed=seed, pop_id=pop_id, NC=NC, NR=NR, fitness=kind, storage=storage,
                       traj_cap=max(gens, 1))
    pop.init_population()
    pop.fitness()
    if mode == "plain":
        pop.step_plain(gens)
    else:
        pop.step(gens)
    pop.sync()
    out = pop.as_int8(), pop.fitness_host(), pop.trajectory()
    pop.close()
    return out


def _run_oracle(m, N, seed, gens, NC=1, NR=1, kind=0, pop_id=0):
    ref = oracle.init_population(m, 4 * N, seed, pop_id)
    F = oracle.fitness(ref, kind)
    _, tf, ts = oracle.run(ref, F, N, NC, NR, kind, seed, pop_id, 0, gens)
    return ref, F, tf, ts


def _assert_same(gpu, ref):
    p, F, (gtf, gts) = gpu
    rp, rF, tf, ts = ref
    assert np.array_equal(F, rF)
    assert np.array_equal(p, rp)
    assert np.array_equal(gtf.astype(np.uint64), tf)
    assert np.array_equal(gts, ts)


@pytest.mark.parametrize("mode", ["plain", "fused"])
@pytest.mark.parametrize("storage", [0, 1])
def test_config1_m12_P1000_200_generations(mode, storage):
    """m = 12, P = 1,000, F_sq, one pair-flip per child, 200 generations, seed 0."""
    h = need_gpu()
    _assert_same(_run_gpu(h, 12, 250, 0, 200, storage, mode), _run_oracle(12, 250, 0, 200))


@pytest.mark.parametrize("mode", ["plain", "fused"])
def test_config2_m20_P40000_prefix(mode):
    """m = 20, P = 40,000 (the paper's scale), seed 1: the first 25 generations."""
    h = need_gpu()
    _assert_same(_run_gpu(h, 20, 10000, 1, 25, 1, mode), _run_oracle(20, 10000, 1, 25))


@pytest.mark.parametrize("mode", ["plain", "fused"])
@pytest.mark.parametrize("m,N,NC,NR,kind", [(4, 1, 1, 1, 0), (8, 3, 2, 2, 2), (16, 40, 4, 2, 1),
                                            (28, 33, 1, 10, 2), (36, 25, 2, 3, 0), (68, 21, 1, 1, 0),
                                            (92, 19, 2, 2, 1), (100, 20, 1, 1, 0), (128, 9, 4, 2, 2)])
def test_small_configs(mode, m, N, NC, NR, kind):
    h = need_gpu()
    _assert_same(_run_gpu(h, m, N, 7, 30, 1, mode, NC, NR, kind, pop_id=3),
                 _run_oracle(m, N, 7, 30, NC, NR, kind, pop_id=3))


def test_fused_kernel_is_used_for_the_paper_scale():
    h = need_gpu()
    pop = h.Population(20, 10000, seed=1, storage=1)
    assert pop.is_fused()
    pop.close()


@pytest.mark.parametrize("storage", [0, 1])
def test_mixed_plain_and_fused_resume(storage):
    """Checkpoint/resume: plain generations, then fused ones, then plain,
    equal one oracle run (the state is population, fitness and g)."""
    h = need_gpu()
    m, N, seed = 16, 300, 9
    pop = h.Population(m, N, seed=seed, NC=2, NR=2, fitness=2, storage=storage, traj_cap=64)
    pop.init_population()
    pop.fitness()
    pop.step_plain(7)
    pop.step(70)           # crosses a chunk boundary of the persistent kernel
    pop.step_plain(3)
    pop.sync()
    assert pop.generation() == 80
    ref = oracle.init_population(m, 4 * N, seed)
    F = oracle.fitness(ref, 2)
    _, tf, ts = oracle.run(ref, F, N, 2, 2, 2, seed, 0, 0, 80)
    assert np.array_equal(pop.as_int8(), ref)
    assert np.array_equal(pop.fitness_host(), F)
    gtf, gts = pop.trajectory()
    assert np.array_equal(gtf.astype(np.uint64), tf[-64:]) and np.array_equal(gts, ts[-64:])


def test_stop_at_zero_finds_order_12_hadamard():
    h = need_gpu()
    m, N, seed, NC, NR = 12, 1000, 3, 2, 2
    ref = oracle.init_population(m, 4 * N, seed)
    F = oracle.fitness(ref, 2)
    n_ref, tf, ts = oracle.run(ref, F, N, NC, NR, 2, seed, 0, 0, 400, stop_at_zero=True)
    pop = h.Population(m, N, seed=seed, NC=NC, NR=NR, fitness=2, storage=1, traj_cap=512)
    pop.init_population()
    pop.fitness()
    done = pop.step(400, stop_at_zero=True)
    assert done == n_ref
    assert np.array_equal(pop.as_int8(), ref)
    if tf[-1] == 0:
        H = pop.get_slot(int(ts[-1])).astype(np.int64)
        assert np.array_equal(H.T @ H, m * np.eye(m, dtype=np.int64))


def test_multi_population_mixed_orders_one_launch():
    """Mixed orders 12..36 in one persistent launch, each population equal
    to its own oracle run (sizes reduced from the 2,000-20,000 range)."""
    h = need_gpu()
    orders = [12, 16, 20, 24, 28, 32, 36]
    pops, refs = [], []
    for idx, m in enumerate(orders):
        N = 40 + 37 * idx
        p = h.Population(m, N, seed=3, pop_id=idx, fitness=0, storage=1, traj_cap=64)
        p.init_population()
        p.fitness()
        pops.append(p)
        r = oracle.init_population(m, 4 * N, 3, idx)
        F = oracle.fitness(r, 0)
        _, tf, ts = oracle.run(r, F, N, 1, 1, 0, 3, idx, 0, 60)
        refs.append((r, F, tf, ts))
    h.step_multi(pops, 60)
    for p, (r, F, tf, ts) in zip(pops, refs):
        p.sync()
        assert p.generation() == 60
        assert np.array_equal(p.as_int8(), r)
        assert np.array_equal(p.fitness_host(), F)
        gtf, gts = p.trajectory()
        assert np.array_equal(gtf.astype(np.uint64), tf) and np.array_equal(gts, ts)


def test_graph_replay_equals_oracle():
    """CUDA-graph replays of 10-generation chunks (device generation
    counters), then a plain remainder, equal the oracle run."""
    h = need_gpu()
    stream = torch.cuda.Stream()
    specs = [(12, 50), (20, 61), (36, 23)]
    pops = []
    for i, (m, N) in enumerate(specs):
        p = h.Population(m, N, seed=4, pop_id=i, fitness=0, storage=1, traj_cap=64, stream=stream)
        p.init_population()
        p.fitness()
        pops.append(p)
    h.step_multi_graph(pops, 35, 10)     # 3 replays of 10 + 5 through ga_step_multi
    for p in pops:
        p.step_plain(2)
    torch.cuda.synchronize()
    for i, ((m, N), p) in enumerate(zip(specs, pops)):
        ref = oracle.init_population(m, 4 * N, 4, i)
        F = oracle.fitness(ref, 0)
        _, tf, ts = oracle.run(ref, F, N, 1, 1, 0, 4, i, 0, 37)
        assert p.generation() == 37
        assert np.array_equal(p.as_int8(), ref)
        assert np.array_equal(p.fitness_host(), F)
        gtf, gts = p.trajectory()
        assert np.array_equal(gtf.astype(np.uint64), tf) and np.array_equal(gts, ts)


def test_fused_grid_setting_does_not_change_results():
    h = need_gpu()
    out = []
    for blocks in (0, 37):
        p = h.Population(20, 700, seed=8, storage=1, traj_cap=16)
        h.set_fused_grid(p, blocks)
        p.init_population()
        p.fitness()
        p.step(16)
        p.sync()
        out.append((p.as_int8(), p.fitness_host()))
        p.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_config2_full_1000_generations_fused():
    """m = 20, P = 40,000, seed 1: all 1,000 generations, fused kernel,
    bit-exact with the oracle (population, fitness, best trajectory)."""
    h = need_gpu()
    gpu = _run_gpu(h, 20, 10000, 1, 1000, 1, "fused")
    _assert_same(gpu, _run_oracle(20, 10000, 1, 1000))


@pytest.mark.parametrize("mode", ["plain", "fused"])
@pytest.mark.parametrize("m,N,NC,NR,kind", [(12, 50, 1, 1, 2), (20, 64, 2, 3, 0), (36, 25, 1, 1, 0),
                                            (100, 12, 3, 2, 1)])
def test_mutation_method1_matches_oracle(mode, m, N, NC, NR, kind):
    """Mutation method 1 of Sec. 3.5 (one draw shared by the generation's
    offspring): plain and fused paths equal the oracle bit for bit."""
    h = need_gpu()
    gens, seed = 12, 8
    pop = h.Population(m, N, seed=seed, NC=NC, NR=NR, fitness=kind, storage=1, traj_cap=gens, mutation=1)
    pop.init_population()
    pop.fitness()
    if mode == "fused":
        pop.step(gens)
    else:
        pop.step_plain(gens)
    pop.sync()
    ref = oracle.init_population(m, 4 * N, seed)
    F = oracle.fitness(ref, kind)
    _, tf, ts = oracle.run(ref, F, N, NC, NR, kind, seed, 0, 0, gens, shared_mutation=1)
    assert np.array_equal(pop.as_int8(), ref)
    assert np.array_equal(pop.fitness_host(), F)
    gtf, gts = pop.trajectory()
    assert np.array_equal(gtf.astype(np.uint64), tf) and np.array_equal(gts, ts)
    pop.close()


def test_fused_m32_P80000_paper_search_parameters():
    """The paper's m = 32 search parameters (Sec. 4.4: P = 80,000, NC = 1,
    NR = 12, F2) in the fused kernel (strict: no fallback), 20 generations,
    bit-exact with the oracle.  2N = 40,000 survivors take the survivor-order
    sort with keys in global memory."""
    h = need_gpu()
    m, N, gens, NC, NR, kind, seed = 32, 20000, 20, 1, 12, 2, 9
    pop = h.Population(m, N, seed=seed, NC=NC, NR=NR, fitness=kind, storage=h.STORE_BITS, traj_cap=gens)
    pop.set_strict(True)
    assert pop.is_fused()
    pop.init_population()
    pop.fitness()
    pop.step(gens)
    pop.sync()
    gpu = pop.as_int8(), pop.fitness_host(), pop.trajectory()
    pop.close()
    _assert_same(gpu, _run_oracle(m, N, seed, gens, NC, NR, kind))


@pytest.mark.parametrize("m,N,gens", [(20, 30000, 12), (64, 16384, 6), (8, 65536, 4)])
def test_fused_large_populations_match_oracle(m, N, gens):
    """Populations whose 2N survivors exceed the shared-memory survivor sort
    (2N > 24,576), up to P = 262,144 at m = 8, fused and strict."""
    h = need_gpu()
    pop = h.Population(m, N, seed=4, storage=h.STORE_BITS, traj_cap=gens)
    pop.set_strict(True)
    pop.init_population()
    pop.fitness()
    pop.step(gens)
    pop.sync()
    gpu = pop.as_int8(), pop.fitness_host(), pop.trajectory()
    pop.close()
    _assert_same(gpu, _run_oracle(m, N, 4, gens))


def test_strict_mode_reports_instead_of_falling_back():
    """m = 256 is beyond the persistent kernel: a strict context reports
    GA_EUNSUPPORTED with the reason; a non-strict one runs the plain path."""
    h = need_gpu()
    pop = h.Population(256, 2, seed=1, storage=h.STORE_BITS, traj_cap=4)
    assert not pop.is_fused()
    with pytest.raises(h.GAError) as ei:
        pop.set_strict(True)
    assert ei.value.status == h.GA_EUNSUPPORTED and "m <= 128" in str(ei.value)
    pop.init_population()
    pop.fitness()
    with pytest.raises(h.GAError) as ei:
        pop.step(2)
    assert ei.value.status == h.GA_EUNSUPPORTED
    pop.set_strict(False)
    pop.step(2)
    pop.sync()
    assert pop.generation() == 2
    pop.close()


@pytest.mark.parametrize("m,N,tpp,nch", [(4, 5, 2, 0), (12, 250, 2, 0), (20, 501, 2, 0), (32, 300, 2, 0), (24, 97, 4, 0),
                                         (40, 200, 0, 1), (64, 150, 0, 7), (100, 60, 0, 16), (128, 40, 0, 3)])
def test_fused_launch_shapes_give_identical_results(m, N, tpp, nch):
    """Every launch shape the autotuner may pick (two or four threads per
    pair at m <= 32; any warp-Gram chunking at m > 32) computes the same
    generations as the oracle."""
    h = need_gpu()
    gens = 9
    pop = h.Population(m, N, seed=21, storage=h.STORE_BITS, traj_cap=gens, NC=2, NR=2, fitness=2)
    h.set_fused_shape(pop, tpp, nch)
    pop.set_strict(True)
    pop.init_population()
    pop.fitness()
    pop.step(gens)
    pop.sync()
    gpu = pop.as_int8(), pop.fitness_host(), pop.trajectory()
    pop.close()
    _assert_same(gpu, _run_oracle(m, N, 21, gens, 2, 2, 2))


def test_mixed_orders_with_tuned_shapes_in_one_launch():
    h = need_gpu()
    specs = [(8, 300, 2, 0), (20, 211, 4, 0), (28, 150, 2, 0), (36, 90, 0, 5), (96, 30, 0, 11)]
    gens = 7
    pops = []
    for i, (m, N, tpp, nch) in enumerate(specs):
        p = h.Population(m, N, seed=8, pop_id=i, storage=h.STORE_BITS, traj_cap=gens)
        h.set_fused_shape(p, tpp, nch)
        p.set_strict(True)
        p.init_population()
        p.fitness()
        pops.append(p)
    h.step_multi(pops, gens)
    for i, ((m, N, _, _), p) in enumerate(zip(specs, pops)):
        p.sync()
        _assert_same((p.as_int8(), p.fitness_host(), p.trajectory()), _run_oracle(m, N, 8, gens, pop_id=i))
        p.close()


def test_auto_path_override_picks_the_measured_path():
    h = need_gpu()
    import torch
    m, P = 32, 4096
    pop = h.empty_population(h.STORE_INT8, m, P)
    h.ga_init_batch(pop, h.STORE_INT8, m, P, 5)
    ref = torch.zeros(P, dtype=torch.int32, device="cuda")
    h.ga_fitness_batch(pop, h.STORE_INT8, m, P, h.FIT_SQ, h.PATH_INT32, ref)
    for path in (h.PATH_POPC, h.PATH_IMMA, h.PATH_INT32):
        h.set_auto_path(h.STORE_INT8, m, h.FIT_SQ, path)
        got = torch.zeros(P, dtype=torch.int32, device="cuda")
        h.ga_fitness_batch(pop, h.STORE_INT8, m, P, h.FIT_SQ, h.PATH_AUTO, got)
        assert torch.equal(got, ref)
    h.set_auto_path(h.STORE_INT8, m, h.FIT_SQ, h.PATH_AUTO)


@pytest.mark.parametrize("m,N,gens", [(64, 64, 6), (100, 40, 4)])
def test_threshold_below_the_histogram_window(m, N, gens):
    """2N - 1 planted Sylvester matrices (F = 0) and random others: the first
    generation's threshold is a random matrix's F, the next one falls to
    the planted copies' offspring, far below the window of exact buckets
    kept under the previous threshold, so the search must take bucket 0 and
    refine from 0.  Bit-exact with the oracle."""
    h = need_gpu()
    from hadamard_fixtures import sylvester
    H = sylvester(64) if m == 64 else None
    pop = h.Population(m, N, seed=17, storage=h.STORE_BITS, traj_cap=gens)
    pop.set_strict(True)
    pop.init_population()
    host = pop.as_int8()
    if H is not None:
        host[:2 * N - 1] = H
    else:
        # m = 100 has no Sylvester matrix: plant copies of the population's best instead
        F0 = oracle.fitness(host, oracle.FIT_SQ)
        host[:2 * N - 1] = host[int(np.argmin(F0))]
    pop.load_int8(host)
    pop.fitness()
    pop.step(gens)
    pop.sync()
    gpu = pop.as_int8(), pop.fitness_host(), pop.trajectory()
    pop.close()
    ref = host.copy()
    F = oracle.fitness(ref, oracle.FIT_SQ)
    _, tf, ts = oracle.run(ref, F, N, 1, 1, oracle.FIT_SQ, 17, 0, 0, gens)
    _assert_same(gpu, (ref, F, tf, ts))


def test_config4_full_sizes_graph_prefix():
    """Config 4 at its real sizes: orders 12..36 with P = 4 (500 + U[0, 4500])
    from the CONFIG stream (seed 3), one persistent launch per CUDA-graph
    chunk of 10 generations, 20 generations, every population equal to its
    own oracle run."""
    h = need_gpu()
    orders = [12, 16, 20, 24, 28, 32, 36]
    gens = 20
    stream = torch.cuda.Stream()
    pops, refs = [], []
    for idx, m in enumerate(orders):
        N = oracle.mixed_N(3, idx)
        p = h.Population(m, N, seed=3, pop_id=idx, fitness=0, storage=1, traj_cap=64, stream=stream)
        p.set_strict(True)
        p.init_population()
        p.fitness()
        pops.append(p)
        r = oracle.init_population(m, 4 * N, 3, idx)
        F = oracle.fitness(r, 0)
        _, tf, ts = oracle.run(r, F, N, 1, 1, 0, 3, idx, 0, gens)
        refs.append((r, F, tf, ts))
    h.step_multi_graph(pops, gens, 10)
    for p, ref in zip(pops, refs):
        p.sync()
        assert p.generation() == gens
        _assert_same((p.as_int8(), p.fitness_host(), p.trajectory()), ref)
        p.close()
