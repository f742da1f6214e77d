// k_ops.cu -- the one-kernel-per-operator path: a5 crossover, a6 mutation,
// a8 best individual, and storage conversion.
#include "common.cuh"
#include "kernels.cuh"

namespace hadga {

// ---------------------------------------------------------------------------
// a5 -- column-exchange crossover (Sec. 3.4, Fig. 2, Eq. (6)).
// Pair k: cut c = U[1, m-1] from (CROSS, gen, k, 0);
//   slot 2N+k = P_k[:, :c] | P_{N+k}[:, c:],  slot 3N+k = P_{N+k}[:, :c] | P_k[:, c:].
// One warp per pair; lane 0 draws c.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_cross_int8(uint32_t *pop, int m, int64_t N, uint32_t seed, uint32_t pop_id,
                                                    uint32_t gen)
{
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int words = (m * m) >> 2, rw = m >> 2;
    for (int64_t k = gw; k < N; k += nw) {
        int c = 0;
        if (lane == 0)
            c = cut_point(seed, pop_id, gen, (uint32_t)k, m);
        c = __shfl_sync(0xFFFFFFFFu, c, 0);
        const uint32_t *p1 = pop + (size_t)k * words, *p2 = pop + (size_t)(N + k) * words;
        uint32_t *o1 = pop + (size_t)(2 * N + k) * words, *o2 = pop + (size_t)(3 * N + k) * words;
        for (int e = lane; e < words; e += 32) {
            // bytes 4*(e % rw) .. +3 of a row are columns j0 .. j0+3
            const int j0 = 4 * (e % rw);
            uint32_t keep = 0;  // byte lanes taken from the first parent
#pragma unroll
            for (int b = 0; b < 4; ++b)
                keep |= (j0 + b < c) ? (0xFFu << (8 * b)) : 0u;
            const uint32_t a = p1[e], bb = p2[e];
            o1[e] = (a & keep) | (bb & ~keep);
            o2[e] = (bb & keep) | (a & ~keep);
        }
    }
}

__global__ void __launch_bounds__(256) k_cross_bits(uint32_t *pop, int m, int W, int64_t N, uint32_t seed,
                                                    uint32_t pop_id, uint32_t gen)
{
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int words = m * W;
    for (int64_t k = gw; k < N; k += nw) {
        int c = 0;
        if (lane == 0)
            c = cut_point(seed, pop_id, gen, (uint32_t)k, m);
        c = __shfl_sync(0xFFFFFFFFu, c, 0);
        const uint32_t *p1 = pop + (size_t)k * words, *p2 = pop + (size_t)(N + k) * words;
        uint32_t *o1 = pop + (size_t)(2 * N + k) * words, *o2 = pop + (size_t)(3 * N + k) * words;
        for (int e = lane; e < words; e += 32) {
            const bool first = (e / W) < c;
            const uint32_t a = p1[e], b = p2[e];
            o1[e] = first ? a : b;
            o2[e] = first ? b : a;
        }
    }
}

cudaError_t launch_crossover(void *pop, int storage, int m, int64_t N, uint32_t seed, uint32_t pop_id, uint32_t gen,
                             cudaStream_t s)
{
    const int bs = 256;
    int64_t grid = (N * 32 + bs - 1) / bs;
    if (grid > 65535)
        grid = 65535;
    if (storage == ST_INT8)
        k_cross_int8<<<(unsigned)grid, bs, 0, s>>>((uint32_t *)pop, m, N, seed, pop_id, gen);
    else if (storage == ST_BITS)
        k_cross_bits<<<(unsigned)grid, bs, 0, s>>>((uint32_t *)pop, m, words_per_col(m), N, seed, pop_id, gen);
    else
        return cudaErrorInvalidValue;
    note_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// a6 -- balanced pair-flip mutation, method 3 (Sec. 3.5, Eq. (7), Fig. 3).
// Offspring o (slot 2N+o): stream (MUTATE, gen, o, 0) gives NC columns in
// [1, m-1], then NR first rows, then NR second rows in [0, m-1].  For each
// column in order and each pair in order the two entries are negated iff
// they differ.  With `shared` (method 1 of Sec. 3.5) every offspring uses
// the draws of stream index 2N.  One thread per offspring, reading the
// stream sequentially.
// ---------------------------------------------------------------------------
struct MutStream {
    uint32_t seed, pop_id, gen, o, block;
    uint4 cur;
    int used;
    __device__ MutStream(uint32_t s, uint32_t p, uint32_t g, uint32_t oo)
        : seed(s), pop_id(p), gen(g), o(oo), block(0), cur(make_uint4(0, 0, 0, 0)), used(4) {}
    __device__ __forceinline__ uint32_t next()
    {
        if (used == 4) {
            cur = philox_block(seed, pop_id, OP_MUTATE, gen, o, 0u, block++);
            used = 0;
        }
        return word_of(cur, used++);
    }
};

template <bool BITS>
__global__ void __launch_bounds__(128) k_mutate(void *pop, int m, int64_t N, int NC, int NR, uint32_t seed,
                                                uint32_t pop_id, uint32_t gen, int shared)
{
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= 2 * N)
        return;
    const int W = words_per_col(m);
    // draws: NC columns, NR first rows, NR second rows (at most 64 each)
    uint8_t col[64], r1[64], r2[64];
    MutStream st(seed, pop_id, gen, shared ? (uint32_t)(2 * N) : (uint32_t)o);
    for (int jc = 0; jc < NC; ++jc)
        col[jc] = (uint8_t)uniform_int(st.next(), 1u, (uint32_t)(m - 1));
    for (int ir = 0; ir < NR; ++ir)
        r1[ir] = (uint8_t)uniform_int(st.next(), 0u, (uint32_t)(m - 1));
    for (int ir = 0; ir < NR; ++ir)
        r2[ir] = (uint8_t)uniform_int(st.next(), 0u, (uint32_t)(m - 1));
    const int64_t slot = 2 * N + o;
    for (int jc = 0; jc < NC; ++jc) {
        const int c = col[jc];
        for (int ir = 0; ir < NR; ++ir) {
            const int a = r1[ir], b = r2[ir];
            if (BITS) {
                uint32_t *cw = (uint32_t *)pop + (size_t)slot * m * W + (size_t)c * W;
                const uint32_t ba = (cw[a >> 5] >> (a & 31)) & 1u, bb = (cw[b >> 5] >> (b & 31)) & 1u;
                if (ba != bb) {
                    cw[a >> 5] ^= 1u << (a & 31);
                    cw[b >> 5] ^= 1u << (b & 31);
                }
            } else {
                int8_t *Q = (int8_t *)pop + (size_t)slot * m * m;
                const int8_t va = Q[a * m + c], vb = Q[b * m + c];
                if (va != vb) {
                    Q[a * m + c] = (int8_t)-va;
                    Q[b * m + c] = (int8_t)-vb;
                }
            }
        }
    }
}

cudaError_t launch_mutate(void *pop, int storage, int m, int64_t N, int NC, int NR, uint32_t seed, uint32_t pop_id,
                          uint32_t gen, int shared, cudaStream_t s)
{
    const int bs = 128;
    const unsigned grid = (unsigned)((2 * N + bs - 1) / bs);
    if (storage == ST_BITS)
        k_mutate<true><<<grid, bs, 0, s>>>(pop, m, N, NC, NR, seed, pop_id, gen, shared);
    else if (storage == ST_INT8)
        k_mutate<false><<<grid, bs, 0, s>>>(pop, m, N, NC, NR, seed, pop_id, gen, shared);
    else
        return cudaErrorInvalidValue;
    note_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// a8 -- least (F << 32 | slot): fitness first, lowest slot on ties.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_best(const uint32_t *__restrict__ fit, int64_t P, unsigned long long *out)
{
    __shared__ unsigned long long s_min[8];
    unsigned long long v = ~0ull;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < P; q += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long key = ((unsigned long long)fit[q] << 32) | (unsigned long long)(uint32_t)q;
        v = key < v ? key : v;
    }
    v = warp_min_u64(v);
    if ((threadIdx.x & 31) == 0)
        s_min[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < (blockDim.x >> 5) ? s_min[threadIdx.x] : ~0ull;
        v = warp_min_u64(v);
        if (threadIdx.x == 0)
            atomicMin(out, v);
    }
}

cudaError_t launch_best(const uint32_t *fit, int64_t P, unsigned long long *out, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(out, 0xFF, sizeof(unsigned long long), s);
    if (e != cudaSuccess)
        return e;
    const int bs = 256;
    int64_t grid = (P + bs - 1) / bs;
    if (grid > 1024)
        grid = 1024;
    k_best<<<(unsigned)grid, bs, 0, s>>>(fit, P, out);
    note_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Storage conversion: one thread per (matrix, column), through bit columns.
// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(256) k_convert(const void *src, int ss, void *dst, int ds, int m, int64_t P)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= P * m)
        return;
    const int64_t q = t / m;
    const int j = (int)(t % m);
    uint32_t v[W];
#pragma unroll
    for (int w = 0; w < W; ++w)
        v[w] = 0u;
    if (ss == ST_BITS) {
        const uint32_t *s = (const uint32_t *)src + (size_t)q * m * W + (size_t)j * W;
#pragma unroll
        for (int w = 0; w < W; ++w)
            v[w] = s[w];
    } else {
        const size_t base = (size_t)q * m * m + j;
        for (int i = 0; i < m; ++i) {
            const size_t e = base + (size_t)i * m;
            bool neg;
            if (ss == ST_INT8)
                neg = ((const int8_t *)src)[e] < 0;
            else if (ss == ST_E4M3)
                neg = (((const uint8_t *)src)[e] & 0x80u) != 0;
            else
                neg = (((const uint16_t *)src)[e] & 0x8000u) != 0;
            if (neg)
                v[i >> 5] |= 1u << (i & 31);
        }
    }
    if (ds == ST_BITS) {
        uint32_t *d = (uint32_t *)dst + (size_t)q * m * W + (size_t)j * W;
#pragma unroll
        for (int w = 0; w < W; ++w)
            d[w] = v[w];
        return;
    }
    const size_t base = (size_t)q * m * m + j;
    for (int i = 0; i < m; ++i) {
        const bool neg = (v[i >> 5] >> (i & 31)) & 1u;
        const size_t e = base + (size_t)i * m;
        if (ds == ST_INT8)
            ((int8_t *)dst)[e] = neg ? (int8_t)-1 : (int8_t)1;
        else if (ds == ST_E4M3)
            ((uint8_t *)dst)[e] = neg ? (uint8_t)0xB8 : (uint8_t)0x38;
        else
            ((uint16_t *)dst)[e] = neg ? (uint16_t)0xBF80 : (uint16_t)0x3F80;
    }
}

cudaError_t launch_convert(const void *src, int src_storage, void *dst, int dst_storage, int m, int64_t P,
                           cudaStream_t s)
{
    if (P <= 0)
        return cudaSuccess;
    const int bs = 256;
    const int64_t grid = (P * m + bs - 1) / bs;
    switch (words_per_col(m)) {
#define HADGA_CV(W)                                                                                          \
    case W:                                                                                                  \
        k_convert<W><<<(unsigned)grid, bs, 0, s>>>(src, src_storage, dst, dst_storage, m, P);                \
        break;
        HADGA_CV(1) HADGA_CV(2) HADGA_CV(3) HADGA_CV(4) HADGA_CV(5) HADGA_CV(6) HADGA_CV(7) HADGA_CV(8)
#undef HADGA_CV
    default:
        return cudaErrorInvalidValue;
    }
    note_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Tiled half-Gram of the incremental mode, recomputed from the bit columns:
// one warp per matrix, a half-warp per 8 x 8 tile, a lane per word of four
// entries (i, j..j+3); 0 where i >= j or outside m.
// ---------------------------------------------------------------------------
template <int W>
__device__ __forceinline__ uint32_t tile_word(const uint32_t *cols, int m, int I, int J, int wi)
{
    const int i = 8 * I + (wi >> 1), j0 = 8 * J + (wi & 1) * 4;
    uint32_t x = 0u;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int j = j0 + k;
        if (i < j && j < m) {
            int d = 0;
#pragma unroll
            for (int w = 0; w < W; ++w)
                d += __popc(cols[i * W + w] ^ cols[j * W + w]);
            x |= ((uint32_t)(m / 2 - d) & 0xFFu) << (8 * k);
        }
    }
    return x;
}

template <int W>
__global__ void __launch_bounds__(256) k_gram_store(const uint32_t *__restrict__ pop, int m, int64_t P, int8_t *gram,
                                                    int dpad, uint32_t *gidx)
{
    extern __shared__ uint32_t s_c[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint32_t *cols = s_c + (size_t)wib * m * W;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int nb = gram_tiles_nb(m), nt = gram_tiles(m);
    for (int64_t q = gw; q < P; q += nw) {
        for (int e = lane; e < m * W; e += 32)
            cols[e] = pop[(size_t)q * m * W + e];
        __syncwarp();
        uint32_t *G = reinterpret_cast<uint32_t *>(gram + (size_t)q * dpad);
        for (int t = lane >> 4; t < nt; t += 2) {
            int I, J;
            tile_coords(t, nb, I, J);
            G[(size_t)t * 16 + (lane & 15)] = tile_word<W>(cols, m, I, J, lane & 15);
        }
        if (lane == 0)
            gidx[q] = (uint32_t)q;
        __syncwarp();
    }
}

cudaError_t launch_gram_store(const uint32_t *pop, int m, int64_t P, int8_t *gram, int dpad, uint32_t *gidx,
                              cudaStream_t s)
{
    const int W = words_per_col(m);
    const int wpb = 8;
    const size_t smem = (size_t)wpb * m * W * 4;
    int64_t grid = (P + wpb - 1) / wpb;
    if (grid > 4096)
        grid = 4096;
    switch (W) {
    case 1: k_gram_store<1><<<(unsigned)grid, wpb * 32, smem, s>>>(pop, m, P, gram, dpad, gidx); break;
    case 2: k_gram_store<2><<<(unsigned)grid, wpb * 32, smem, s>>>(pop, m, P, gram, dpad, gidx); break;
    case 3: k_gram_store<3><<<(unsigned)grid, wpb * 32, smem, s>>>(pop, m, P, gram, dpad, gidx); break;
    case 4: k_gram_store<4><<<(unsigned)grid, wpb * 32, smem, s>>>(pop, m, P, gram, dpad, gidx); break;
    default: return cudaErrorInvalidValue;
    }
    note_launches(1);
    return cudaGetLastError();
}

// Full recomputation check: every stored word against the recomputed one
// (counted per word that differs), and every fitness word against the sum
// of the recomputed terms.
template <int W>
__global__ void __launch_bounds__(256) k_gram_check(const uint32_t *__restrict__ pop, int m, int64_t P, int kind,
                                                    const int8_t *__restrict__ gram, int dpad,
                                                    const uint32_t *__restrict__ gidx, const uint32_t *__restrict__ fit,
                                                    unsigned long long *counts)
{
    extern __shared__ uint32_t s_c[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint32_t *cols = s_c + (size_t)wib * m * W;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int nb = gram_tiles_nb(m), nt = gram_tiles(m);
    unsigned long long bad_e = 0, bad_f = 0;
    for (int64_t q = gw; q < P; q += nw) {
        for (int e = lane; e < m * W; e += 32)
            cols[e] = pop[(size_t)q * m * W + e];
        __syncwarp();
        const uint32_t gq = gidx[q];
        const bool in_range = (int64_t)gq < P;
        const uint32_t *G = reinterpret_cast<const uint32_t *>(gram + (size_t)(in_range ? gq : 0u) * dpad);
        uint32_t acc = 0;
        for (int t = lane >> 4; t < nt; t += 2) {
            int I, J;
            tile_coords(t, nb, I, J);
            const uint32_t x = tile_word<W>(cols, m, I, J, lane & 15);
            acc += (uint32_t)(kind == FIT_SQ ? word_terms<FIT_SQ>(x)
                                             : kind == FIT_ABS ? word_terms<FIT_ABS>(x) : word_terms<FIT_NNZ>(x));
            if (!in_range || G[(size_t)t * 16 + (lane & 15)] != x)
                ++bad_e;
        }
        acc = warp_sum(acc);
        const uint32_t f = kind == FIT_SQ ? word_terms_finish<FIT_SQ>(acc)
                                          : kind == FIT_ABS ? word_terms_finish<FIT_ABS>(acc)
                                                            : word_terms_finish<FIT_NNZ>(acc);
        if (lane == 0 && f != fit[q])
            ++bad_f;
        __syncwarp();
    }
    for (int o = 16; o > 0; o >>= 1) {
        bad_e += __shfl_xor_sync(0xFFFFFFFFu, bad_e, o);
        bad_f += __shfl_xor_sync(0xFFFFFFFFu, bad_f, o);
    }
    if (lane == 0 && (bad_e | bad_f)) {
        atomicAdd(counts, bad_e);
        atomicAdd(counts + 1, bad_f);
    }
}

cudaError_t launch_gram_check(const uint32_t *pop, int m, int64_t P, int kind, const int8_t *gram, int dpad,
                              const uint32_t *gidx, const uint32_t *fit, unsigned long long *counts, cudaStream_t s)
{
    const int W = words_per_col(m);
    const int wpb = 8;
    const size_t smem = (size_t)wpb * m * W * 4;
    int64_t grid = (P + wpb - 1) / wpb;
    if (grid > 4096)
        grid = 4096;
    switch (W) {
    case 1: k_gram_check<1><<<(unsigned)grid, wpb * 32, smem, s>>>(pop, m, P, kind, gram, dpad, gidx, fit, counts); break;
    case 2: k_gram_check<2><<<(unsigned)grid, wpb * 32, smem, s>>>(pop, m, P, kind, gram, dpad, gidx, fit, counts); break;
    case 3: k_gram_check<3><<<(unsigned)grid, wpb * 32, smem, s>>>(pop, m, P, kind, gram, dpad, gidx, fit, counts); break;
    case 4: k_gram_check<4><<<(unsigned)grid, wpb * 32, smem, s>>>(pop, m, P, kind, gram, dpad, gidx, fit, counts); break;
    default: return cudaErrorInvalidValue;
    }
    note_launches(1);
    return cudaGetLastError();
}

} // namespace hadga
