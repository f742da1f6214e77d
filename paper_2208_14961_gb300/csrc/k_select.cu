// k_select.cu -- a3 truncation selection and a4 random placement of the
// survivors (Sec. 3.3; Sec. 6, the selection line), one kernel per step.
//
// Survivors are the 2N slots first in ascending (F, slot) order.  Instead
// of sorting all P keys, the threshold T (the 2N-th smallest F) is found by
// a three-level radix select over the 32-bit fitness (11 + 11 + 10 bits);
// then every F < T survives together with the lowest `take_eq` slots with
// F == T.  Per tile of 32 slots two ballot masks (F < T, F == T) give, after
// one scan over tiles, the survivors in slot order s_0 < ... < s_{2N-1}.
// Parent slot p receives s_{pi(p)}, pi sorting the Philox keys (u_d, d).
#include "common.cuh"
#include "kernels.cuh"

namespace hadga {

namespace {
constexpr int kRadixBuckets = 2048;
__host__ __device__ constexpr int level_shift(int l) { return l == 0 ? 21 : (l == 1 ? 10 : 0); }
__host__ __device__ constexpr int level_bits(int l) { return l == 2 ? 10 : 11; }
} // namespace

// Histogram of the level-l digit of every F whose higher digits match the
// prefix found so far.
__global__ void __launch_bounds__(1024) k_sel_hist(const uint32_t *__restrict__ fit, int64_t P, int level,
                                                   const SelState *st, uint32_t *hist)
{
    __shared__ uint32_t s_h[kRadixBuckets];
    for (int i = threadIdx.x; i < kRadixBuckets; i += blockDim.x)
        s_h[i] = 0u;
    __syncthreads();
    const int sh = level_shift(level), nb = level_bits(level);
    const int hs = sh + nb;  // bits above this level
    const uint32_t pre = level == 0 ? 0u : (st->prefix >> hs);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < P; q += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t f = fit[q];
        if (level == 0 || (f >> hs) == pre)
            atomicAdd(&s_h[(f >> sh) & ((1u << nb) - 1u)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kRadixBuckets; i += blockDim.x)
        if (s_h[i])
            atomicAdd(&hist[i], s_h[i]);
}

// One block: finds the digit whose cumulative count reaches `need`, extends
// the prefix, and clears the histogram for the next level.
__global__ void __launch_bounds__(1024) k_sel_pick(uint32_t *hist, int level, SelState *st, uint32_t n_keep,
                                                   uint32_t *err)
{
    __shared__ uint32_t tmp[33];
    __shared__ uint32_t s_found;
    const int sh = level_shift(level);
    const uint32_t need = level == 0 ? n_keep : st->need;
    if (threadIdx.x == 0)
        s_found = 0u;
    uint32_t carry = 0;
    for (int base = 0; base < kRadixBuckets; base += blockDim.x) {
        const int b = base + threadIdx.x;
        const uint32_t h = b < kRadixBuckets ? hist[b] : 0u;
        uint32_t total;
        const uint32_t ex = block_excl_scan(h, tmp, &total) + carry;
        if (b < kRadixBuckets && h > 0u && ex < need && need <= ex + h) {
            const uint32_t pre = level == 0 ? 0u : st->prefix;
            st->prefix = pre | ((uint32_t)b << sh);
            st->need = need - ex;
            s_found = 1u;
        }
        carry += total;
        __syncthreads();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (!s_found)
            atomicOr(err, ERR_INTERNAL);
        else if (level == 2) {
            st->T = st->prefix;
            st->take_eq = st->need;
        }
    }
    for (int b = threadIdx.x; b < kRadixBuckets; b += blockDim.x)
        hist[b] = 0u;
}

// One warp per tile of 32 slots: masks of F < T and F == T.
__global__ void __launch_bounds__(256) k_sel_tiles(const uint32_t *__restrict__ fit, int64_t P, const SelState *st,
                                                   unsigned long long *tmask)
{
    const int lane = threadIdx.x & 31;
    const int64_t tiles = (P + 31) >> 5;
    const uint32_t T = st->T;
    for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < tiles;
         t += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t q = t * 32 + lane;
        const uint32_t f = q < P ? fit[q] : 0u;
        const uint32_t lt = __ballot_sync(0xFFFFFFFFu, q < P && f < T);
        const uint32_t eq = __ballot_sync(0xFFFFFFFFu, q < P && f == T);
        if (lane == 0)
            tmask[t] = (unsigned long long)lt | ((unsigned long long)eq << 32);
    }
}

// One block: survivor mask of every tile and the number of survivors in the
// tiles before it.
__global__ void __launch_bounds__(1024) k_sel_scan(const unsigned long long *__restrict__ tmask, int64_t tiles,
                                                   const SelState *st, uint32_t n_keep, uint32_t *survmask,
                                                   uint32_t *survbefore, uint32_t *err)
{
    __shared__ uint32_t tmp[33];
    const uint32_t take = st->take_eq;
    uint32_t eq_carry = 0, sv_carry = 0, total;
    for (int64_t base = 0; base < tiles; base += blockDim.x) {
        const int64_t t = base + threadIdx.x;
        const unsigned long long tm = t < tiles ? tmask[t] : 0ull;
        const uint32_t lt = (uint32_t)tm, eq = (uint32_t)(tm >> 32);
        const uint32_t eqb = block_excl_scan((uint32_t)__popc(eq), tmp, &total) + eq_carry;
        eq_carry += total;
        const int keep = take > eqb ? (int)(take - eqb) : 0;
        const uint32_t sm = lt | lowest_set_bits(eq, keep);
        const uint32_t svb = block_excl_scan((uint32_t)__popc(sm), tmp, &total) + sv_carry;
        sv_carry += total;
        if (t < tiles) {
            survmask[t] = sm;
            survbefore[t] = svb;
        }
    }
    if (threadIdx.x == 0 && sv_carry != n_keep)
        atomicOr(err, ERR_INTERNAL);
}

// ---------------------------------------------------------------------------
// a4 -- survivor order pi of one generation, one block.  Keys
// ((u_d << 32) | d) are counted into 2^nbits buckets by their top bits,
// scattered bucket by bucket, and ranked inside their bucket by counting
// smaller keys; pi[rank] = d.  One Philox block (SELECT, gen, t) gives the
// keys of d = 4t .. 4t+3.  With G > 0 a thread keeps the blocks of its
// groups t = tid + i * blockDim (i < G) in registers between the counting
// and the scattering pass (the caller guarantees ceil(n / 4) <= G * blockDim);
// with G = 0 they are drawn again.
// ---------------------------------------------------------------------------
template <int G>
__device__ void perm_block(uint32_t n, uint32_t seed, uint32_t pop_id, uint32_t gen, uint32_t *out,
                           unsigned long long *keys, uint32_t *cnt, uint32_t *off, int nbits, uint32_t *tmp)
{
    const uint32_t B = 1u << nbits;
    const int sh = 32 - nbits;
    const uint32_t ngroups = (n + 3u) >> 2;
    constexpr int GR = G > 0 ? G : 1;
    uint4 kb[GR];
    for (uint32_t b = threadIdx.x; b < B; b += blockDim.x)
        cnt[b] = 0u;
    __syncthreads();
    if (G > 0) {
#pragma unroll
        for (int i = 0; i < GR; ++i) {
            const uint32_t t = threadIdx.x + (uint32_t)i * blockDim.x;
            if (t < ngroups) {
                kb[i] = philox_block(seed, pop_id, OP_SELECT, gen, t, 0u, 0u);
#pragma unroll
                for (int w = 0; w < 4; ++w)
                    if (4u * t + w < n)
                        atomicAdd(&cnt[word_of(kb[i], w) >> sh], 1u);
            }
        }
    } else {
        for (uint32_t t = threadIdx.x; t < ngroups; t += blockDim.x) {
            const uint4 b = philox_block(seed, pop_id, OP_SELECT, gen, t, 0u, 0u);
#pragma unroll
            for (int w = 0; w < 4; ++w)
                if (4u * t + w < n)
                    atomicAdd(&cnt[word_of(b, w) >> sh], 1u);
        }
    }
    __syncthreads();
    uint32_t carry = 0, total;
    for (uint32_t base = 0; base < B; base += blockDim.x) {
        const uint32_t b = base + threadIdx.x;
        const uint32_t c = b < B ? cnt[b] : 0u;
        const uint32_t ex = block_excl_scan(c, tmp, &total) + carry;
        carry += total;
        if (b < B) {
            off[b] = ex;
            cnt[b] = ex;  // becomes the scatter cursor
        }
    }
    __syncthreads();
    auto scatter = [&](uint32_t t, const uint4 &b) {
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const uint32_t d = 4u * t + w;
            if (d < n) {
                const uint32_t u = word_of(b, w);
                const uint32_t pos = atomicAdd(&cnt[u >> sh], 1u);
                keys[pos] = ((unsigned long long)u << 32) | d;
            }
        }
    };
    if (G > 0) {
#pragma unroll
        for (int i = 0; i < GR; ++i) {
            const uint32_t t = threadIdx.x + (uint32_t)i * blockDim.x;
            if (t < ngroups)
                scatter(t, kb[i]);
        }
    } else {
        for (uint32_t t = threadIdx.x; t < ngroups; t += blockDim.x)
            scatter(t, philox_block(seed, pop_id, OP_SELECT, gen, t, 0u, 0u));
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
        const unsigned long long k = keys[i];
        const uint32_t b = (uint32_t)(k >> 32) >> sh;
        const uint32_t lo = off[b], hi = cnt[b];
        uint32_t r = 0;
        for (uint32_t j = lo; j < hi; ++j)
            r += keys[j] < k ? 1u : 0u;
        out[lo + r] = (uint32_t)k;
    }
    __syncthreads();
}

// Philox groups a thread of the 1024-thread shared-memory sort keeps in
// registers: ceil(kPermSmemMax / 4) <= kPermGroups * 1024.
constexpr int kPermGroups = 6;
static_assert(kPermSmemMax <= 4u * kPermGroups * 1024u, "survivor-order groups exceed the register buffer");

__global__ void __launch_bounds__(1024) k_perm_smem(uint32_t n, uint32_t seed, uint32_t pop_id, uint32_t gen0,
                                                    uint32_t *out, const uint32_t *gen_dev)
{
    extern __shared__ __align__(16) unsigned long long s_keys[];
    __shared__ uint32_t s_cnt[1 << kPermSmemBits], s_off[1 << kPermSmemBits], s_tmp[33];
    const uint32_t g0 = gen_dev ? *gen_dev + 1u : gen0;
    perm_block<kPermGroups>(n, seed, pop_id, g0 + blockIdx.x, out + (size_t)blockIdx.x * n, s_keys, s_cnt, s_off,
                            kPermSmemBits, s_tmp);
}

__global__ void k_set_u32(uint32_t *p, uint32_t v) { *p = v; }

cudaError_t launch_set_u32(uint32_t *p, uint32_t v, cudaStream_t s)
{
    k_set_u32<<<1, 1, 0, s>>>(p, v);
    note_launches(1);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(1024) k_perm_global(uint32_t n, uint32_t seed, uint32_t pop_id, uint32_t gen,
                                                      uint32_t *out, unsigned long long *keys, uint32_t *cnt,
                                                      int nbits)
{
    __shared__ uint32_t s_tmp[33];
    perm_block<0>(n, seed, pop_id, gen, out, keys, cnt, cnt + (1u << nbits), nbits, s_tmp);
}

// Survivor orders of `gridDim.x` consecutive generations for n > kPermSmemMax
// (one block per generation): bucket counters and offsets in shared memory
// (2^nbits buckets each), the keys of generation b in keys[b * n .. ),
// Philox blocks drawn twice.  The result is the full sort of the keys, the
// same as the shared-memory sort's.
__global__ void __launch_bounds__(1024) k_perm_big(uint32_t n, uint32_t seed, uint32_t pop_id, uint32_t gen0,
                                                   uint32_t *out, unsigned long long *keys, int nbits,
                                                   const uint32_t *gen_dev)
{
    extern __shared__ __align__(16) uint32_t s_cnt_off[];
    __shared__ uint32_t s_tmp[33];
    const uint32_t g0 = gen_dev ? *gen_dev + 1u : gen0;
    const uint32_t B = 1u << nbits;
    perm_block<0>(n, seed, pop_id, g0 + blockIdx.x, out + (size_t)blockIdx.x * n, keys + (size_t)blockIdx.x * n,
                  s_cnt_off, s_cnt_off + B, nbits, s_tmp);
}

// Buckets of k_perm_big: about eight keys per bucket, at most 2^kPermBigMaxBits
// (the counters and offsets then take 2 * 4 * 2^14 = 128 KiB of shared memory).
constexpr int kPermBigMaxBits = 14;

int perm_big_bits(uint32_t n)
{
    int b = 0;
    while ((1u << b) < n)
        ++b;
    b -= 3;
    return b < kPermSmemBits ? kPermSmemBits : (b > kPermBigMaxBits ? kPermBigMaxBits : b);
}

int perm_global_bits(uint32_t n)
{
    int b = 0;
    while ((1u << b) < n)
        ++b;
    b -= 3;  // about eight keys per bucket
    return b < kPermSmemBits ? kPermSmemBits : (b > 24 ? 24 : b);
}

cudaError_t launch_perm_table(uint32_t n, uint32_t seed, uint32_t pop_id, uint32_t gen0, int ngen, uint32_t *out,
                              cudaStream_t s, const uint32_t *gen_dev, unsigned long long *keys)
{
    if (ngen <= 0)
        return cudaErrorInvalidValue;
    if (n > kPermSmemMax) {
        if (!keys)
            return cudaErrorInvalidValue;
        const int nb = perm_big_bits(n);
        const size_t smem = (size_t)2u * (1u << nb) * sizeof(uint32_t);
        cudaError_t e = cudaFuncSetAttribute(k_perm_big, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
        k_perm_big<<<ngen, 1024, smem, s>>>(n, seed, pop_id, gen0, out, keys, nb, gen_dev);
        note_launches(1);
        return cudaGetLastError();
    }
    const size_t smem = (size_t)n * sizeof(unsigned long long);
    cudaError_t e = cudaFuncSetAttribute(k_perm_smem, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kPermSmemMax * sizeof(unsigned long long)));
    if (e != cudaSuccess)
        return e;
    k_perm_smem<<<ngen, 1024, smem, s>>>(n, seed, pop_id, gen0, out, gen_dev);
    note_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Gather of the parents: warp per parent slot p.  Survivor pi(p) is found by
// a binary search over the tile prefix counts and a select-bit in its tile.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t survivor_slot(uint32_t d, const uint32_t *survmask, const uint32_t *survbefore,
                                                 int64_t tiles)
{
    int64_t lo = 0, hi = tiles - 1;  // largest t with survbefore[t] <= d
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (survbefore[mid] <= d)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo * 32 + nth_set_bit(survmask[lo], (int)(d - survbefore[lo]));
}

__global__ void __launch_bounds__(256) k_sel_gather(const uint8_t *__restrict__ pop, const uint32_t *__restrict__ fit,
                                                    size_t mat_bytes, int64_t n_keep, const uint32_t *perm,
                                                    const uint32_t *survmask, const uint32_t *survbefore,
                                                    int64_t tiles, int64_t P, uint8_t *out_pop, uint32_t *out_fit,
                                                    uint32_t *err)
{
    const int lane = threadIdx.x & 31;
    for (int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < n_keep;
         p += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        int64_t src = 0;
        if (lane == 0) {
            src = survivor_slot(perm[p], survmask, survbefore, tiles);
            if (src >= P) {  // only if the survivor masks were inconsistent
                atomicOr(err, ERR_INTERNAL);
                src = P - 1;
            }
            out_fit[p] = fit[src];
        }
        src = __shfl_sync(0xFFFFFFFFu, src, 0);
        const uint4 *a = reinterpret_cast<const uint4 *>(pop + (size_t)src * mat_bytes);
        uint4 *b = reinterpret_cast<uint4 *>(out_pop + (size_t)p * mat_bytes);
        for (size_t e = lane; e < mat_bytes / 16; e += 32)
            b[e] = a[e];
    }
}

// ---------------------------------------------------------------------------
// Probabilistic selection (the Sec. 3.3 variant, weights inverse to F): one
// warp per tile writes the in-tile weight prefixes and the tile sum; one
// block scans the tile sums; one warp per parent slot draws and gathers.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_psel_tiles(const uint32_t *__restrict__ fit, int64_t P,
                                                    unsigned long long *cw, unsigned long long *tsum)
{
    const int lane = threadIdx.x & 31;
    const int64_t tiles = (P + 31) >> 5;
    for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < tiles;
         t += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t q = t * 32 + lane;
        const uint32_t f = q < P ? fit[q] : 0u;
        const unsigned long long sum = psel_tile(f, q < P, cw + (size_t)t * 32u, lane);
        if (lane == 0)
            tsum[t] = sum;
    }
}

// One block: exclusive prefix of the tile sums and their total.
__global__ void __launch_bounds__(1024) k_psel_scan(const unsigned long long *__restrict__ tsum, int64_t tiles,
                                                    unsigned long long *tex, unsigned long long *total)
{
    __shared__ unsigned long long s_w[32];
    __shared__ unsigned long long s_tot;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned long long carry = 0;
    for (int64_t base = 0; base < tiles; base += blockDim.x) {
        const int64_t t = base + threadIdx.x;
        const unsigned long long v = t < tiles ? tsum[t] : 0ull;
        unsigned long long inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
            if (lane >= o)
                inc += y;
        }
        if (lane == 31)
            s_w[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            const unsigned long long x = lane < nw ? s_w[lane] : 0ull;
            unsigned long long xi = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, xi, o);
                if (lane >= o)
                    xi += y;
            }
            if (lane < nw)
                s_w[lane] = xi - x;  // exclusive prefix of the warp totals
        }
        __syncthreads();
        const unsigned long long ex = carry + s_w[warp] + inc - v;
        if (t < tiles)
            tex[t] = ex;
        // the chunk's total: the last thread's inclusive value
        if (threadIdx.x == blockDim.x - 1)
            s_tot = ex + v;
        __syncthreads();
        carry = s_tot;
        __syncthreads();
    }
    if (threadIdx.x == 0)
        *total = carry;
}

__global__ void __launch_bounds__(256) k_psel_gather(const uint8_t *__restrict__ pop,
                                                     const uint32_t *__restrict__ fit, size_t mat_bytes,
                                                     int64_t n_keep, const unsigned long long *tex,
                                                     const unsigned long long *cw, const unsigned long long *total,
                                                     int64_t tiles, int64_t P, uint32_t seed, uint32_t pop_id,
                                                     uint32_t gen, uint8_t *out_pop, uint32_t *out_fit, uint32_t *err)
{
    const int lane = threadIdx.x & 31;
    const unsigned long long W = *total;
    for (int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < n_keep;
         p += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        uint32_t src = 0;
        if (lane == 0) {
            const unsigned long long u = psel_draw(seed, pop_id, gen, (uint32_t)p);
            src = psel_lookup(u, [&](uint32_t j) { return tex[j]; }, (uint32_t)tiles, 0ull, W, cw, (uint32_t)P, err);
            out_fit[p] = fit[src];
        }
        src = __shfl_sync(0xFFFFFFFFu, src, 0);
        const uint4 *a = reinterpret_cast<const uint4 *>(pop + (size_t)src * mat_bytes);
        uint4 *b = reinterpret_cast<uint4 *>(out_pop + (size_t)p * mat_bytes);
        for (size_t e = lane; e < mat_bytes / 16; e += 32)
            b[e] = a[e];
    }
}

cudaError_t launch_select_prob(const void *pop, const uint32_t *fit, int64_t N, size_t mat_bytes, uint32_t seed,
                               uint32_t pop_id, uint32_t gen, const SelWork &w, void *scratch_pop,
                               uint32_t *scratch_fit, cudaStream_t s)
{
    const int64_t P = 4 * N, n_keep = 2 * N, tiles = (P + 31) / 32;
    int64_t tg = (tiles * 32 + 255) / 256;
    if (tg > 4096)
        tg = 4096;
    k_psel_tiles<<<(unsigned)tg, 256, 0, s>>>(fit, P, w.cw, w.tmask);
    k_psel_scan<<<1, 1024, 0, s>>>(w.tmask, tiles, w.tex, w.wtotal);
    int64_t gg = (n_keep * 32 + 255) / 256;
    if (gg > 8192)
        gg = 8192;
    k_psel_gather<<<(unsigned)gg, 256, 0, s>>>((const uint8_t *)pop, fit, mat_bytes, n_keep, w.tex, w.cw, w.wtotal,
                                               tiles, P, seed, pop_id, gen, (uint8_t *)scratch_pop, scratch_fit,
                                               w.err);
    note_launches(3);
    return cudaGetLastError();
}

cudaError_t launch_select(const void *pop, const uint32_t *fit, int64_t N, size_t mat_bytes, uint32_t seed,
                          uint32_t pop_id, uint32_t gen, const SelWork &w, void *scratch_pop, uint32_t *scratch_fit,
                          cudaStream_t s)
{
    const int64_t P = 4 * N, n_keep = 2 * N, tiles = (P + 31) / 32;
    int64_t grid = (P + 1023) / 1024;
    if (grid > 256)
        grid = 256;
    for (int level = 0; level < 3; ++level) {
        k_sel_hist<<<(unsigned)grid, 1024, 0, s>>>(fit, P, level, w.state, w.hist);
        k_sel_pick<<<1, 1024, 0, s>>>(w.hist, level, w.state, (uint32_t)n_keep, w.err);
    }
    int64_t tg = (tiles * 32 + 255) / 256;
    if (tg > 4096)
        tg = 4096;
    k_sel_tiles<<<(unsigned)tg, 256, 0, s>>>(fit, P, w.state, w.tmask);
    k_sel_scan<<<1, 1024, 0, s>>>(w.tmask, tiles, w.state, (uint32_t)n_keep, w.survmask, w.survbefore, w.err);
    cudaError_t e;
    if ((uint64_t)n_keep <= kPermSmemMax) {
        e = launch_perm_table((uint32_t)n_keep, seed, pop_id, gen, 1, w.perm, s);
    } else {
        const int nb = perm_global_bits((uint32_t)n_keep);
        k_perm_global<<<1, 1024, 0, s>>>((uint32_t)n_keep, seed, pop_id, gen, w.perm, w.perm_keys, w.perm_cnt, nb);
        note_launches(1);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess)
        return e;
    int64_t gg = (n_keep * 32 + 255) / 256;
    if (gg > 8192)
        gg = 8192;
    k_sel_gather<<<(unsigned)gg, 256, 0, s>>>((const uint8_t *)pop, fit, mat_bytes, n_keep, w.perm, w.survmask,
                                              w.survbefore, tiles, P, (uint8_t *)scratch_pop, scratch_fit, w.err);
    note_launches(9);  // 3 x (histogram, pick), tiles, scan, gather
    return cudaGetLastError();
}

} // namespace hadga
