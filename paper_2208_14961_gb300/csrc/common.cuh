// common.cuh -- device helpers shared by the libhadga kernels (sm_103a).
//
// Randomness follows Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel
// Random Numbers: As Easy as 1, 2, 3", SC'11): ten rounds of two
// 32x32->64-bit multiplies with the key bumped by the Weyl constants between
// rounds.  Key (seed, pop_id); counter (op, generation, index,
// (sub << 16) | block).  A word w maps to [lo, hi] as
// lo + floor(w * (hi - lo + 1) / 2^32).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace hadga {

enum : uint32_t { OP_INIT = 0, OP_SELECT = 1, OP_CROSS = 2, OP_MUTATE = 3, OP_PSELECT = 5 };
enum : uint32_t { ERR_TIMEOUT = 1u, ERR_INTERNAL = 2u };
enum { FIT_SQ = 0, FIT_ABS = 1, FIT_NNZ = 2 };
enum { ST_INT8 = 0, ST_BITS = 1, ST_E4M3 = 2, ST_BF16 = 3 };

// Upper bound on the order m; the bit storage uses W = ceil(m/32) <= 8 words.
constexpr int kMaxM = 256;
constexpr int kMaxW = 8;

__host__ __device__ __forceinline__ int words_per_col(int m) { return (m + 31) >> 5; }

// ---------------------------------------------------------------------------
// Philox4x32-10
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t lo_a = 0xD2511F53u * c.x, hi_a = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo_b = 0xCD9E8D57u * c.z, hi_b = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi_b ^ c.y ^ k.x, lo_b, hi_a ^ c.w ^ k.y, lo_a);
    }
    return c;
}

__device__ __forceinline__ uint4 philox_block(uint32_t seed, uint32_t pop_id, uint32_t op, uint32_t gen,
                                              uint32_t index, uint32_t sub, uint32_t block)
{
    return philox10(make_uint4(op, gen, index, (sub << 16) | block), make_uint2(seed, pop_id));
}

__device__ __forceinline__ uint32_t word_of(const uint4 &v, int i)
{
    return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}

// Integer in [lo, hi] from one word (span hi - lo + 1 < 2^32).
__device__ __forceinline__ uint32_t uniform_int(uint32_t w, uint32_t lo, uint32_t hi)
{
    return lo + __umulhi(w, hi - lo + 1u);
}

// Key u_d of the survivor order of generation `gen`: word (d mod 4) of
// Philox block (SELECT, gen, floor(d/4), 0).
__device__ __forceinline__ uint32_t select_key(uint32_t seed, uint32_t pop_id, uint32_t gen, uint32_t d)
{
    const uint4 b = philox_block(seed, pop_id, OP_SELECT, gen, d >> 2, 0u, 0u);
    return word_of(b, d & 3);
}

// Cut point of pair k at generation gen: U[1, m-1] from (CROSS, gen, k, 0).
__device__ __forceinline__ int cut_point(uint32_t seed, uint32_t pop_id, uint32_t gen, uint32_t k, int m)
{
    const uint4 b = philox_block(seed, pop_id, OP_CROSS, gen, k, 0u, 0u);
    return (int)uniform_int(b.x, 1u, (uint32_t)(m - 1));
}

// ---------------------------------------------------------------------------
// Probabilistic selection (the Sec. 3.3 variant: probabilities inverse to the
// fitness).  Weight w = floor(2^32 / (F + 1)); parent slot p draws the 64-bit
// u of words 0, 1 of Philox (PSELECT, gen, p, 0) and takes the individual
// whose cumulative-weight interval holds t = floor(u W / 2^64).
// ---------------------------------------------------------------------------
// floor(2^32 / d) for d = f + 1 in 32-bit arithmetic: floor((2^32 - 1) / d),
// plus one when d divides 2^32 (d a power of two); 2^32 for f = 0.
__device__ __forceinline__ unsigned long long psel_weight(uint32_t f)
{
    if (f == 0u)
        return 1ull << 32;
    const uint32_t d = f + 1u;
    if (d == 0u)  // f = 2^32 - 1 (never a fitness value): 2^32 / 2^32
        return 1ull;
    return (unsigned long long)(0xFFFFFFFFu / d + ((d & (d - 1u)) == 0u ? 1u : 0u));
}

__device__ __forceinline__ unsigned long long psel_draw(uint32_t seed, uint32_t pop_id, uint32_t gen, uint32_t p)
{
    const uint4 b = philox_block(seed, pop_id, OP_PSELECT, gen, p, 0u, 0u);
    return ((unsigned long long)b.x << 32) | (unsigned long long)b.y;
}

// Whole warp, one tile of 32 slots (lane = slot - 32 t): stores the inclusive
// prefix of the tile's weights at cw_tile[lane] (slots past the population
// weigh 0, so their entries equal the tile sum) and returns the tile's sum.
__device__ __forceinline__ unsigned long long psel_tile(uint32_t f, bool valid, unsigned long long *cw_tile, int lane)
{
    unsigned long long w = valid ? psel_weight(f) : 0ull;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xFFFFFFFFu, w, o);
        if (lane >= o)
            w += t;
    }
    cw_tile[lane] = w;
    return __shfl_sync(0xFFFFFFFFu, w, 31);
}

// Slot drawn by u: t = base + floor(u W / 2^64); the tile j is the last with
// ex_at(j) <= t (ex_at: exclusive prefix of the tile sums, from base), the
// slot inside it the first whose inclusive in-tile prefix exceeds t - ex_at(j).
template <class ExAt>
__device__ __forceinline__ uint32_t psel_lookup(unsigned long long u, ExAt ex_at, uint32_t ntiles,
                                                unsigned long long base, unsigned long long W,
                                                const unsigned long long *cw, uint32_t P, uint32_t *err)
{
    const unsigned long long t = base + __umul64hi(u, W);
    uint32_t lo = 0, hi = ntiles - 1u;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1u) >> 1;
        if (ex_at(mid) <= t)
            lo = mid;
        else
            hi = mid - 1u;
    }
    const unsigned long long r = t - ex_at(lo);
    const uint4 *c4 = reinterpret_cast<const uint4 *>(cw + (size_t)lo * 32u);
    uint32_t cnt = 0;
#pragma unroll
    for (int v = 0; v < 16; ++v) {
        const uint4 x = __ldcg(c4 + v);
        const unsigned long long a = ((unsigned long long)x.y << 32) | x.x, b = ((unsigned long long)x.w << 32) | x.z;
        cnt += (a <= r ? 1u : 0u) + (b <= r ? 1u : 0u);
    }
    const uint32_t slot = lo * 32u + cnt;
    if (cnt >= 32u || slot >= P) {  // only if the prefixes were inconsistent
        atomicOr(err, ERR_INTERNAL);
        return P - 1u;
    }
    return slot;
}

// ---------------------------------------------------------------------------
// Bits
// ---------------------------------------------------------------------------
// Position (0-based) of the n-th (0-based) set bit of x; requires n < popc(x).
__device__ __forceinline__ int nth_set_bit(uint32_t x, int n)
{
    int pos = 0;
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const int c = __popc(x & ((1u << w) - 1u));
        if (n >= c) {
            n -= c;
            x >>= w;
            pos += w;
        }
    }
    return pos;
}

// Mask of the lowest `keep` set bits of x (keep <= popc(x)).
__device__ __forceinline__ uint32_t lowest_set_bits(uint32_t x, int keep)
{
    if (keep <= 0)
        return 0u;
    if (keep >= __popc(x))
        return x;
    const int p = nth_set_bit(x, keep - 1);
    return x & (p == 31 ? 0xFFFFFFFFu : ((2u << p) - 1u));
}

// Per-pair fitness term of G = m - 2 d (d = rows where the columns differ).
template <int KIND>
__device__ __forceinline__ uint32_t fit_term(int g)
{
    if (KIND == FIT_SQ)
        return (uint32_t)(g * g);
    if (KIND == FIT_ABS)
        return (uint32_t)(g < 0 ? -g : g);
    return g != 0 ? 1u : 0u;
}

// Sums of terms over i < j become the fitness: F_sq as is, F1 and F2 count
// both triangles (the diagonal contributes |m| - m = 0 and 1 - 1 = 0 per
// entry after subtracting m^2, respectively m).
template <int KIND>
__device__ __forceinline__ uint32_t fit_finish(uint32_t upper_sum)
{
    return KIND == FIT_SQ ? upper_sum : 2u * upper_sum;
}

// ---------------------------------------------------------------------------
// Warp / block reductions and scans
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t warp_sum(uint32_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xFFFFFFFFu, v, o);
        v = t < v ? t : v;
    }
    return v;
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, v, o);
        if (lane >= o)
            v += t;
    }
    return v;
}

// Exclusive scan of one value per thread over the whole block; `tmp` holds
// at least 33 words of shared memory.  Returns the exclusive prefix; *total
// (all threads) receives the block sum.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *tmp, uint32_t *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    const uint32_t inc = warp_incl_scan(v, lane);
    if (lane == 31)
        tmp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = lane < nw ? tmp[lane] : 0u;
        const uint32_t wi = warp_incl_scan(w, lane);
        if (lane < nw)
            tmp[lane] = wi - w;
        if (lane == 31)
            tmp[32] = wi;
    }
    __syncthreads();
    const uint32_t res = tmp[warp] + inc - v;
    *total = tmp[32];
    __syncthreads();
    return res;
}

// ---------------------------------------------------------------------------
// Warp-level fitness of one matrix whose bit columns (W words each) sit in
// shared memory (warp_fitness_cols below).
// ---------------------------------------------------------------------------
// One column of W words from shared memory with the widest aligned vector
// loads (consecutive lanes reading consecutive columns stay bank-conflict
// free; `col` is 4W-byte aligned when W is even).
template <int W>
__device__ __forceinline__ void load_col(const uint32_t *col, uint32_t (&c)[W])
{
    if (W % 4 == 0) {
#pragma unroll
        for (int v = 0; v < W / 4; ++v) {
            const uint4 x = reinterpret_cast<const uint4 *>(col)[v];
            c[4 * v] = x.x, c[4 * v + 1] = x.y, c[4 * v + 2] = x.z, c[4 * v + 3] = x.w;
        }
    } else if (W % 2 == 0) {
#pragma unroll
        for (int v = 0; v < W / 2; ++v) {
            const uint2 x = reinterpret_cast<const uint2 *>(col)[v];
            c[2 * v] = x.x, c[2 * v + 1] = x.y;
        }
    } else {
#pragma unroll
        for (int w = 0; w < W; ++w)
            c[w] = col[w];
    }
}

// Carry-save adder: per bit, a + b + c = s + 2 * carry.
__device__ __forceinline__ void csa(uint32_t a, uint32_t b, uint32_t c, uint32_t &s, uint32_t &carry)
{
    s = a ^ b ^ c;
    carry = (a & b) | (c & (a | b));
}

// Rows where two bit columns differ, d = popc(a ^ b) over W words.  For
// W >= 3 groups of three XOR words go through a carry-save adder first
// (Harley and Seal's population-count method): popc(x0) + popc(x1) +
// popc(x2) = popc(s) + 2 popc(carry), so W = 3, 4, 5 take W - 1 population
// counts, W = 6, 7 take W - 2 and W = 8 takes 5 (a third adder joins the two
// sums and x6).  The count is exact.  The population count unit issues at a
// quarter of the integer ALU rate, so one adder (two logic operations)
// per saved count pays.
template <int W>
__device__ __forceinline__ int xor_popc(const uint32_t (&a)[W], const uint32_t (&b)[W])
{
    uint32_t x[W];
#pragma unroll
    for (int k = 0; k < W; ++k)
        x[k] = a[k] ^ b[k];
    if constexpr (W >= 3 && W <= 5) {
        uint32_t s0, c0;
        csa(x[0], x[1], x[2], s0, c0);
        int d = __popc(s0) + 2 * __popc(c0);
#pragma unroll
        for (int k = 3; k < W; ++k)
            d += __popc(x[k]);
        return d;
    } else if constexpr (W >= 6 && W <= 7) {
        uint32_t s0, c0, s1, c1;
        csa(x[0], x[1], x[2], s0, c0);
        csa(x[3], x[4], x[5], s1, c1);
        int d = __popc(s0) + __popc(s1) + 2 * (__popc(c0) + __popc(c1));
        if constexpr (W == 7)
            d += __popc(x[6]);
        return d;
    } else if constexpr (W == 8) {
        uint32_t s0, c0, s1, c1, s2, c2;
        csa(x[0], x[1], x[2], s0, c0);
        csa(x[3], x[4], x[5], s1, c1);
        csa(s0, s1, x[6], s2, c2);
        return __popc(s2) + __popc(x[7]) + 2 * (__popc(c0) + __popc(c1) + __popc(c2));
    } else {
        int d = 0;
#pragma unroll
        for (int w = 0; w < W; ++w)
            d += __popc(x[w]);
        return d;
    }
}

// Chunks per column of the warp-level Gram below: column a's pairs
// (a, a + s mod m), s = 1..m/2, are split into `nch` runs of consecutive s
// so that the m * nch work units spread evenly over the 32 lanes (cost of
// a choice: rounds * (run length + 2), the 2 standing for the per-unit
// set-up).  Evaluated once per kernel (or on the host), not per matrix.
__host__ __device__ __forceinline__ int warp_gram_chunks(int m)
{
    const int half = m >> 1;
    int best = 1, best_cost = 0x7FFFFFFF;
    for (int n = 1; n <= 16 && n <= half; ++n) {
        const int rounds = (m * n + 31) >> 5, run = (half + n - 1) / n;
        const int cost = rounds * (run + 2);
        if (cost < best_cost) {
            best_cost = cost;
            best = n;
        }
    }
    return best;
}

// A column set in shared memory holds the m bit columns followed by copies
// of columns 0 .. m/2 - 2 (column m + j equals column j), so that the pairs
// (a, a + s mod m), s <= m/2, of the warp-level Gram below read columns
// a + s without wrapping: every lane runs the same trip count.
__host__ __device__ __forceinline__ int col_set_cols(int m) { return m + m / 2; }

// Words of a column set of order m with W words per column.
__host__ __device__ __forceinline__ int col_set_words(int m, int W)
{
    return W <= 4 ? col_set_cols(m) * W : col_set_cols(m) * 4 * ((W + 3) / 4);
}

// Word w of column j of a column set.  W <= 4: column j at words
// [jW, jW + W).  W > 4: planes of four words (plane p holds words 4p .. 4p+3
// of every column, mc = col_set_cols(m) columns per plane), so that lanes
// reading consecutive columns issue 16-byte loads at a 16-byte stride (no
// bank conflicts).
template <int W>
__device__ __forceinline__ int col_word_index(int j, int w, int mc)
{
    return W <= 4 ? j * W + w : (w >> 2) * 4 * mc + j * 4 + (w & 3);
}

template <int W>
__device__ __forceinline__ void load_col_any(const uint32_t *cols, int j, int mc, uint32_t (&c)[W])
{
    if constexpr (W <= 4) {
        load_col<W>(cols + j * W, c);
    } else {
#pragma unroll
        for (int p = 0; p < (W + 3) / 4; ++p) {
            const uint4 x = reinterpret_cast<const uint4 *>(cols + p * 4 * mc)[j];
            c[4 * p] = x.x;
            if (4 * p + 1 < W)
                c[(4 * p + 1) % W] = x.y;
            if (4 * p + 2 < W)
                c[(4 * p + 2) % W] = x.z;
            if (4 * p + 3 < W)
                c[(4 * p + 3) % W] = x.w;
        }
    }
}

// Stores word w of column j of a column set, and of its copy m + j.
template <int W>
__device__ __forceinline__ void store_col_word(uint32_t *cols, int j, int w, int m, uint32_t v)
{
    const int mc = col_set_cols(m);
    cols[col_word_index<W>(j, w, mc)] = v;
    if (j < (m >> 1) - 1)
        cols[col_word_index<W>(j + m, w, mc)] = v;
}

// Every unordered pair once: pairs (a, a + s) for s = 1..m/2 (column a + s
// >= m is the copy of column a + s - m), the s = m/2 pair only when
// a < m/2.  Work units (run r of column a) are enumerated run-major, so
// consecutive lanes read consecutive columns.  nch = warp_gram_chunks(m).
template <int W, int KIND>
__device__ __forceinline__ uint32_t warp_fitness_cols(const uint32_t *cols, int m, int lane, int nch)
{
    uint32_t acc = 0;
    const int half = m >> 1, mc = col_set_cols(m);
    const int run = (half + nch - 1) / nch, units = m * nch;
    int r = 0, a = lane;
    while (a >= m) {
        a -= m;
        ++r;
    }
    for (int u = lane; u < units; u += 32) {
        const int s0 = r * run + 1;
        const int s1 = min(s0 + run - 1, a < half ? half : half - 1);
        uint32_t ca[W];
        load_col_any<W>(cols, a, mc, ca);
#pragma unroll 4
        for (int b = a + s0; b <= a + s1; ++b) {
            uint32_t cb[W];
            load_col_any<W>(cols, b, mc, cb);
            acc += fit_term<KIND>(m - 2 * xor_popc<W>(ca, cb));
        }
        a += 32;
        while (a >= m) {
            a -= m;
            ++r;
        }
    }
    return fit_finish<KIND>(warp_sum(acc));
}

// ---------------------------------------------------------------------------
// Asynchronous global -> shared copies (cp.async; 16 bytes through L2 only,
// 4 or 8 bytes through L1) and their commit / wait groups.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
}

template <int BYTES>
__device__ __forceinline__ void cp_async_small(void *smem_dst, const void *gmem_src)
{
    static_assert(BYTES == 4 || BYTES == 8, "cp.async.ca copies 4, 8 or 16 bytes");
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(gmem_src), "n"(BYTES) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

// Waits until at most N of this thread's most recent cp.async groups are
// pending (all older ones complete).
template <int N>
__device__ __forceinline__ void cp_async_wait_group()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// ---------------------------------------------------------------------------
// Tiled half-Gram storage of the incremental fitness mode: H = G / 2 as int8
// in 8 x 8 tiles (I <= J) of the upper triangle, tile t = I nb - I(I-1)/2 +
// (J - I), nb = ceil(m / 8); entry (i, j) at byte 64 t + 8 (i mod 8) +
// (j mod 8); entries with i >= j or outside m are 0.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ int gram_tiles_nb(int m) { return (m + 7) >> 3; }
__host__ __device__ __forceinline__ int gram_tiles(int m) { return gram_tiles_nb(m) * (gram_tiles_nb(m) + 1) / 2; }

// Tile-row I and tile-column J of tile t (tile-row I holds nb - I tiles).
__host__ __device__ __forceinline__ void tile_coords(int t, int nb, int &I, int &J)
{
    const float b = (float)(2 * nb + 1);
    int i = (int)((b - sqrtf(b * b - 8.0f * (float)t)) * 0.5f);
    i = i < 0 ? 0 : (i > nb - 1 ? nb - 1 : i);
    while (i > 0 && i * nb - (i * (i - 1)) / 2 > t)
        --i;
    while (i + 1 < nb && (i + 1) * nb - ((i + 1) * i) / 2 <= t)
        ++i;
    I = i;
    J = i + (t - (i * nb - (i * (i - 1)) / 2));
}

// Sum over the four int8 entries h of a word of the fitness term of G = 2h,
// before the final scale (F_sq = 4 sum h^2, F1 = 4 sum |h|, F2 = 2 sum [h != 0]).
template <int KIND>
__device__ __forceinline__ int word_terms(uint32_t x)
{
    if (KIND == FIT_SQ)
        return __dp4a((int)x, (int)x, 0);
    if (KIND == FIT_ABS)
        return __dp4a((int)__vabsss4(x), 0x01010101, 0);
    return __dp4a((int)__vsetne4(x, 0u), 0x01010101, 0);
}

template <int KIND>
__device__ __forceinline__ uint32_t word_terms_finish(uint32_t sum)
{
    return KIND == FIT_NNZ ? 2u * sum : 4u * sum;
}

// ---------------------------------------------------------------------------
// Bounded waits
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_gpu_add(uint32_t *p, uint32_t v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ---------------------------------------------------------------------------
// mbarriers (completion of asynchronous copies and tensor-core work)
// ---------------------------------------------------------------------------
constexpr unsigned long long kMbarWaitBudgetNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}

// Bounded wait for the phase of `bar` with parity `parity`; false when the
// budget (`budget_ns`, about two seconds unless a test asks for less) ran
// out, or another thread raised an error and the phase is still open (a
// completed phase always reports true).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t *err,
                                          unsigned long long budget_ns = kMbarWaitBudgetNs)
{
    if (mbar_test(bar, parity))
        return true;
    const unsigned long long t0 = global_ns();
    for (uint32_t i = 1;; ++i) {
        if (mbar_test(bar, parity))
            return true;
        if ((i & 255u) == 0u) {
            if (ld_acquire_gpu(err) != 0u)
                return mbar_test(bar, parity);
            if (global_ns() - t0 > budget_ns) {
                atomicOr(err, ERR_TIMEOUT);
                return mbar_test(bar, parity);
            }
        }
    }
}


// Grid-wide barrier for a cooperative launch with every block resident.
// `bar` counts arrivals monotonically (zeroed before the launch); `epoch`
// is the caller's barrier count.  Arrival is a gpu-scope release reduction
// (cumulative over the block's writes ordered by the preceding bar.sync);
// thread 0 then polls with acquire loads under a bounded
// budget of about two seconds; when it runs out, or another block has
// already raised an error, ERR_TIMEOUT is recorded and every block returns
// false so the kernel can exit cleanly instead of hanging.  Callers read
// data written by other blocks through L2 (ld.global.cg or atomics).
constexpr unsigned long long kBarrierBudgetNs = 2000000000ull;

// Split form of the grid barrier: grid_arrive after the block's writes,
// work that needs nothing from other blocks, then grid_wait.
__device__ __forceinline__ void grid_arrive(uint32_t *bar)
{
    __syncthreads();
    // the block's writes precede this release through the bar.sync above
    if (threadIdx.x == 0)
        red_release_gpu_add(bar, 1u);
}

__device__ __forceinline__ bool grid_wait(uint32_t *bar, uint32_t nblocks, uint32_t &epoch, uint32_t *err,
                                          unsigned long long budget_ns = kBarrierBudgetNs)
{
    __shared__ int s_ok;
    epoch += 1u;
    if (threadIdx.x == 0) {
        const uint32_t target = epoch * nblocks;
        int ok = 1;
        const unsigned long long t0 = global_ns();
        uint32_t spins = 0;
        for (;;) {
            const uint32_t v = ld_acquire_gpu(bar);
            if ((int32_t)(v - target) >= 0)
                break;
            if ((++spins & 63u) == 0u) {
                if (ld_acquire_gpu(err) != 0u) {
                    ok = 0;
                    break;
                }
                if (global_ns() - t0 > budget_ns) {
                    atomicOr(err, ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ bool grid_barrier(uint32_t *bar, uint32_t nblocks, uint32_t &epoch, uint32_t *err,
                                             unsigned long long budget_ns = kBarrierBudgetNs)
{
    __shared__ int s_ok;
    __syncthreads();
    epoch += 1u;
    if (threadIdx.x == 0) {
        const uint32_t target = epoch * nblocks;
        // the block's writes precede this release through the bar.sync above
        red_release_gpu_add(bar, 1u);
        int ok = 1;
        const unsigned long long t0 = global_ns();
        uint32_t spins = 0;
        for (;;) {
            const uint32_t v = ld_acquire_gpu(bar);
            if ((int32_t)(v - target) >= 0)
                break;
            if ((++spins & 63u) == 0u) {
                if (ld_acquire_gpu(err) != 0u) {
                    ok = 0;
                    break;
                }
                if (global_ns() - t0 > budget_ns) {
                    atomicOr(err, ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

} // namespace hadga
