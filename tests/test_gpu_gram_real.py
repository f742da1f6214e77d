"""GPU parity of the batched real Gram G_b = Q_b^T Q_b (Sec. 2, Table 1)
against the oracle, through the C ABI.

Tolerance.  Both sides sum the m products of an entry in floating point: the
kernel in the input's precision u_T with one fused multiply-add per term, the
oracle in double.  Each lies within gamma_m(u) * S_ij of the exact value,
S_ij = sum_r |Q_ri Q_rj| and gamma_n(u) = n u / (1 - n u) (Higham, Sec. 3.1),
so |kernel - oracle| <= (gamma_m(u_T) + gamma_m(2^-53)) * S_ij, with S taken
from the oracle's Gram of |Q| (relative error below 1e-13, covered by the
factor 1.001)."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import need_gpu
from hadamard_fixtures import sylvester
from inputs import signed_real, uniform_real

pytestmark = pytest.mark.gpu

U = {torch.float64: 2.0 ** -53, torch.float32: 2.0 ** -24}


def gamma(n, u):
    return n * u / (1.0 - n * u)


def bound(Qnp, dtype):
    m = Qnp.shape[-1]
    S = oracle.gram_real(np.abs(Qnp.astype(np.float64)))
    return 1.001 * (gamma(m, U[dtype]) + gamma(m, 2.0 ** -53)) * S


def run_gpu(h, Qnp, dtype):
    q = torch.as_tensor(Qnp).to(device="cuda", dtype=dtype).contiguous()
    g = torch.full_like(q, float("nan"))
    h.ga_gram_real_batch(q, g)
    torch.cuda.synchronize()
    return g.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("m,B", [(1, 5), (3, 7), (4, 9), (7, 5), (32, 6), (66, 3), (100, 11), (129, 2), (256, 2)])
@pytest.mark.parametrize("gen", [uniform_real, signed_real])
def test_matches_oracle_within_the_summation_bound(dtype, m, B, gen):
    h = need_gpu()
    Q = gen(B, m, 10 + m, np.float64 if dtype == torch.float64 else np.float32)
    G = run_gpu(h, Q, dtype)
    ref = oracle.gram_real(Q)
    assert np.all(np.abs(G - ref) <= bound(Q, dtype))


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("m", [1, 2, 4, 8, 16, 32, 64, 128, 256])
def test_sylvester_is_exact(dtype, m):
    """+-1 products and integer sums below 2^24 are exact in both types."""
    h = need_gpu()
    Q = np.stack([sylvester(m), -sylvester(m)]).astype(np.float64)
    G = run_gpu(h, Q, dtype)
    assert np.array_equal(G, np.broadcast_to(m * np.eye(m), G.shape))


def test_table1_size_sampled_and_symmetric():
    """N = 10,000 matrices of order 100 in float64 (the size of Table 1):
    the whole output is symmetric and finite, and 48 sampled matrices match
    the oracle within the bound."""
    h = need_gpu()
    N, m = 10000, 100
    Q = uniform_real(N, m, 7)
    q = torch.as_tensor(Q).cuda()
    g = torch.empty_like(q)
    h.ga_gram_real_batch(q, g)
    torch.cuda.synchronize()
    assert torch.equal(g, g.transpose(1, 2))
    assert bool(torch.isfinite(g).all())
    idx = np.random.default_rng(8).choice(N, 48, replace=False)
    idx = np.concatenate([idx, [0, N - 1]])
    Gs = g[torch.as_tensor(idx, device="cuda")].cpu().numpy()
    Qs = Q[idx]
    assert np.all(np.abs(Gs - oracle.gram_real(Qs)) <= bound(Qs, torch.float64))


def test_empty_batch_is_a_no_op():
    h = need_gpu()
    q = torch.zeros((0, 8, 8), dtype=torch.float64, device="cuda")
    g = torch.zeros((0, 8, 8), dtype=torch.float64, device="cuda")
    h.ga_gram_real_batch(q, g)
    torch.cuda.synchronize()
