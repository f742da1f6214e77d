// k_init.cu -- a1, the initial population (Sec. 3.1; Sec. 6, population
// set-up and the column-shuffle kernel).
//
// One thread per (slot, column).  The column is held as bits (bit i set iff
// row i is -1): rows 0..m/2-1 start at -1, rows m/2..m-1 at +1, then a
// Fisher-Yates pass swaps entry i1 with i1 + U[0, m-1-i1] for i1 = 0..m-2,
// the draws being the words of Philox stream (INIT, 0, slot, j) in order.
// Column 0 stays all +1.  The column is then written in the requested
// storage; consecutive threads write consecutive columns, so a row of the
// row-major formats is written by adjacent threads.
#include "common.cuh"
#include "kernels.cuh"

namespace hadga {

template <int W>
__device__ __forceinline__ void swap_bits(uint32_t (&v)[W], int i1, int i2)
{
    if (W == 1) {
        const uint32_t t = ((v[0] >> i1) ^ (v[0] >> i2)) & 1u;
        v[0] ^= (t << i1) | (t << i2);
    } else {
        const uint32_t t = ((v[i1 >> 5] >> (i1 & 31)) ^ (v[i2 >> 5] >> (i2 & 31))) & 1u;
        v[i1 >> 5] ^= t << (i1 & 31);
        v[i2 >> 5] ^= t << (i2 & 31);
    }
}

template <int W>
__global__ void __launch_bounds__(256) k_init(void *pop, int storage, int m, int64_t first, int64_t count,
                                              uint32_t seed, uint32_t pop_id)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count * m)
        return;
    const int64_t slot = first + t / m;
    const int j = (int)(t % m);

    uint32_t v[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
        // rows [32w, 32w + 32) that fall below m/2 start at -1
        const int lo = 32 * w, hi = min(32 * w + 32, m / 2);
        const int n = hi > lo ? hi - lo : 0;
        v[w] = (j == 0 || n == 0) ? 0u : (n == 32 ? 0xFFFFFFFFu : ((1u << n) - 1u));
    }
    if (j > 0) {
        int i1 = 0;
        uint32_t block = 0;
        while (i1 < m - 1) {
            const uint4 r = philox_block(seed, pop_id, OP_INIT, 0u, (uint32_t)slot, (uint32_t)j, block++);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (i1 < m - 1) {
                    const int i2 = i1 + (int)uniform_int(word_of(r, q), 0u, (uint32_t)(m - 1 - i1));
                    swap_bits<W>(v, i1, i2);
                    ++i1;
                }
            }
        }
    }

    if (storage == ST_BITS) {
        uint32_t *dst = (uint32_t *)pop + (size_t)slot * m * W + (size_t)j * W;
#pragma unroll
        for (int w = 0; w < W; ++w)
            dst[w] = v[w];
        return;
    }
    const size_t base = (size_t)slot * m * m + (size_t)j;
    for (int i = 0; i < m; ++i) {
        const bool neg = (v[i >> 5] >> (i & 31)) & 1u;
        const size_t e = base + (size_t)i * m;
        if (storage == ST_INT8)
            ((int8_t *)pop)[e] = neg ? (int8_t)-1 : (int8_t)1;
        else if (storage == ST_E4M3)
            ((uint8_t *)pop)[e] = neg ? (uint8_t)0xB8 : (uint8_t)0x38;
        else
            ((uint16_t *)pop)[e] = neg ? (uint16_t)0xBF80 : (uint16_t)0x3F80;
    }
}

cudaError_t launch_init(void *pop, int storage, int m, int64_t first, int64_t count, uint32_t seed, uint32_t pop_id,
                        cudaStream_t s)
{
    if (count <= 0)
        return cudaSuccess;
    const int64_t threads = count * m;
    const int bs = 256;
    const int64_t grid = (threads + bs - 1) / bs;
    switch (words_per_col(m)) {
#define HADGA_INIT_CASE(W)                                                                                   \
    case W:                                                                                                  \
        k_init<W><<<(unsigned)grid, bs, 0, s>>>(pop, storage, m, first, count, seed, pop_id);                \
        break;
        HADGA_INIT_CASE(1)
        HADGA_INIT_CASE(2)
        HADGA_INIT_CASE(3)
        HADGA_INIT_CASE(4)
        HADGA_INIT_CASE(5)
        HADGA_INIT_CASE(6)
        HADGA_INIT_CASE(7)
        HADGA_INIT_CASE(8)
#undef HADGA_INIT_CASE
    default:
        return cudaErrorInvalidValue;
    }
    note_launches(1);
    return cudaGetLastError();
}

} // namespace hadga
