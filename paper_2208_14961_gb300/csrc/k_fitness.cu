// k_fitness.cu -- a2, batched column Gram G = Q^T Q and the fitness reduced
// from its off-diagonal entries (Sec. 3.2, Eq. (3)-(5); Sec. 4.2, Eq. (8)-(9)).
//
// All paths are exact integer computations:
//  * POPC  -- bit storage: G_ij = m - 2 popc(b_i ^ b_j), where b_j holds the
//             -1 rows of column j.  m <= 32: one thread per matrix with the
//             columns in registers; larger m: one warp per matrix, columns
//             staged in shared memory, lane a owning columns a, a + 32, ...
//  * POPC on int8 storage -- one warp per matrix; the sign bits of 32 rows
//             become one column word per __ballot_sync, then as above.
//  * INT32 -- int8 storage, CUDA-core 4-way byte dot products (__dp4a) on a
//             transposed copy in shared memory.
//  * IMMA  -- int8 storage, warp-level mma.sync m16n8k32 on the same
//             transposed copy (both Gram operands read Q^T with the row index
//             contiguous); the int8 signs are turned into FP8 e4m3 operands
//             (+-1 exact) and accumulated in FP32, exact for |G| <= 256.
//  * FP8_WARP -- e4m3 storage, the same warp-level MMA reading the stored
//             bytes directly (shared-memory tiles, cp.async double buffering).
// The pairs i < j of a warp's matrix are enumerated without a table: lane
// a pairs column a with (a + s) mod m for s = 1 .. m/2, the s = m/2 pair only
// when a < m/2, which visits each unordered pair exactly once.
#include "common.cuh"
#include "kernels.cuh"

namespace hadga {

// ---------------------------------------------------------------------------
// POPC, bit storage, m <= 32: one thread per matrix
// ---------------------------------------------------------------------------
template <int M, int KIND>
__global__ void __launch_bounds__(128) k_fit_bits_thread(const uint32_t *__restrict__ pop, int64_t first,
                                                         int64_t count, uint32_t *__restrict__ fit)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count)
        return;
    const int64_t q = first + t;
    const uint4 *src = reinterpret_cast<const uint4 *>(pop + (size_t)q * M);
    uint32_t c[M];
#pragma unroll
    for (int v = 0; v < M / 4; ++v) {
        const uint4 x = __ldg(src + v);
        c[4 * v + 0] = x.x;
        c[4 * v + 1] = x.y;
        c[4 * v + 2] = x.z;
        c[4 * v + 3] = x.w;
    }
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < M; ++i) {
#pragma unroll
        for (int j = i + 1; j < M; ++j)
            acc += fit_term<KIND>(M - 2 * __popc(c[i] ^ c[j]));
    }
    fit[q] = fit_finish<KIND>(acc);
}

template <int W, int KIND>
__global__ void __launch_bounds__(256) k_fit_bits_warp(const uint32_t *__restrict__ pop, int m, int64_t first,
                                                       int64_t count, uint32_t *__restrict__ fit)
{
    extern __shared__ uint32_t s_cols[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint32_t *cols = s_cols + (size_t)wib * col_set_words(m, W);
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int words = m * W, nch = warp_gram_chunks(m);
    for (int64_t q = first + gw; q < first + count; q += nw) {
        const uint32_t *src = pop + (size_t)q * words;
        for (int e = lane; e < words; e += 32)
            store_col_word<W>(cols, e / W, e % W, m, __ldg(src + e));
        __syncwarp();
        const uint32_t f = warp_fitness_cols<W, KIND>(cols, m, lane, nch);
        if (lane == 0)
            fit[q] = f;
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// POPC on int8 storage: sign bits -> column words by ballot
// ---------------------------------------------------------------------------
// Builds the W-word bit columns of an int8 row-major matrix in `cols`
// (column-set layout of col_word_index).
template <int W>
__device__ __forceinline__ void int8_to_cols(const int8_t *Q, int m, uint32_t *cols, int lane)
{
    for (int rg = 0; rg < W; ++rg) {
        const int r = rg * 32 + lane;
        const uint32_t *row = reinterpret_cast<const uint32_t *>(Q + (size_t)r * m);
        for (int cw = 0; cw < (m >> 2); ++cw) {
            const uint32_t x = r < m ? __ldg(row + cw) : 0u;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t bal = __ballot_sync(0xFFFFFFFFu, (x >> (8 * k + 7)) & 1u);
                const int j = 4 * cw + k;
                if (lane == (j & 31))
                    cols[col_word_index<W>(j, rg, col_set_cols(m))] = bal;
            }
        }
    }
}

template <int W, int KIND>
__global__ void __launch_bounds__(256) k_fit_int8_popc(const int8_t *__restrict__ pop, int m, int64_t first,
                                                       int64_t count, uint32_t *__restrict__ fit)
{
    extern __shared__ uint32_t s_cols[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint32_t *cols = s_cols + (size_t)wib * col_set_words(m, W);
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int nch = warp_gram_chunks(m);
    const int mc = col_set_cols(m), ncopy = ((m >> 1) - 1) * W;
    for (int64_t q = first + gw; q < first + count; q += nw) {
        int8_to_cols<W>(pop + (size_t)q * m * m, m, cols, lane);
        __syncwarp();
        // copies of columns 0 .. m/2 - 2 after column m - 1
        for (int e = lane; e < ncopy; e += 32)
            cols[col_word_index<W>(m + e / W, e % W, mc)] = cols[col_word_index<W>(e / W, e % W, mc)];
        __syncwarp();
        const uint32_t f = warp_fitness_cols<W, KIND>(cols, m, lane, nch);
        if (lane == 0)
            fit[q] = f;
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Transposed int8 copy in shared memory: T[j][r] = Q[r][j], row stride
// `ts` bytes (kpad + 16, kpad = m rounded up to 32; padding is zero).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void int8_transpose_to_smem(const int8_t *Q, int m, int mpad, int kpad, int ts,
                                                       int8_t *T, int lane)
{
    // zero the whole tile (padding rows / columns must contribute nothing)
    uint32_t *T32 = reinterpret_cast<uint32_t *>(T);
    for (int e = lane; e < (mpad * ts) >> 2; e += 32)
        T32[e] = 0u;
    __syncwarp();
    const int words = (m * m) >> 2;
    const uint32_t *src = reinterpret_cast<const uint32_t *>(Q);
    for (int e = lane; e < words; e += 32) {
        const uint32_t x = __ldg(src + e);
        const int r = (4 * e) / m, j0 = (4 * e) % m;
#pragma unroll
        for (int k = 0; k < 4; ++k)
            T[(j0 + k) * ts + r] = (int8_t)(x >> (8 * k));
    }
    (void)kpad;
    __syncwarp();
}

template <int KIND>
__global__ void __launch_bounds__(128) k_fit_int8_dp4a(const int8_t *__restrict__ pop, int m, int64_t first,
                                                       int64_t count, uint32_t *__restrict__ fit)
{
    extern __shared__ __align__(16) int8_t s_t[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int kpad = (m + 31) & ~31, mpad = (m + 15) & ~15, ts = kpad + 16;
    int8_t *T = s_t + (size_t)wib * mpad * ts;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int half = m >> 1, kw = m >> 2;
    for (int64_t q = first + gw; q < first + count; q += nw) {
        int8_transpose_to_smem(pop + (size_t)q * m * m, m, mpad, kpad, ts, T, lane);
        uint32_t acc = 0;
        for (int a = lane; a < m; a += 32) {
            const int *ra = reinterpret_cast<const int *>(T + a * ts);
            const int smax = a < half ? half : half - 1;
            int b = a;
            for (int s = 1; s <= smax; ++s) {
                b = (b + 1 == m) ? 0 : b + 1;
                const int *rb = reinterpret_cast<const int *>(T + b * ts);
                int g = 0;
                for (int k = 0; k < kw; ++k)
                    g = __dp4a(ra[k], rb[k], g);
                acc += fit_term<KIND>(g);
            }
        }
        const uint32_t f = fit_finish<KIND>(warp_sum(acc));
        if (lane == 0)
            fit[q] = f;
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Warp-level tensor-core MMA on +-1 data:
// mma.sync.aligned.m16n8k32.row.col.f32.e4m3.e4m3.f32.  +-1 is exact in FP8
// e4m3 (0x38 / 0xB8) and every Gram entry (|G| <= 256) is exact in the FP32
// accumulator.  On this GPU the FP8 form of the warp-level MMA issues at
// about 14x the rate of the int8 (s8) form (peaks microbenchmark: 1.09 P vs
// 76 T multiply-adds/s), so int8 +-1 storage is fed to it through a sign
// conversion: byte x in {0x01, 0xFF} -> 0x38 | (x & 0x80).
// A (16x32, row) and B (32x8, col) registers hold 4 consecutive k elements.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mma_e4m3_16832(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile("mma.sync.aligned.m16n8k32.row.col.f32.e4m3.e4m3.f32 "
                 "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Four int8 +-1 entries -> four e4m3 +-1 entries.
__device__ __forceinline__ uint32_t i8pm1_to_e4m3(uint32_t x) { return (x & 0x80808080u) | 0x38383838u; }

// The same, keeping zero bytes (padding) zero.
__device__ __forceinline__ uint32_t i8_to_e4m3_z(uint32_t x)
{
    return ((x & 0x80808080u) | 0x38383838u) & __vcmpne4(x, 0u);
}

// Operand register of the row-Gram kernels: int8 storage converted, e4m3
// storage as is.
template <bool E4M3>
__device__ __forceinline__ uint32_t fp8_operand(uint32_t x)
{
    return E4M3 ? x : i8pm1_to_e4m3(x);
}

__device__ __forceinline__ int gram_value(float d) { return __float2int_rn(d); }

template <int KIND>
__global__ void __launch_bounds__(128) k_fit_int8_imma(const int8_t *__restrict__ pop, int m, int64_t first,
                                                       int64_t count, uint32_t *__restrict__ fit)
{
    extern __shared__ __align__(16) int8_t s_t[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int kpad = (m + 31) & ~31, mpad = (m + 15) & ~15, ts = kpad + 16;
    int8_t *T = s_t + (size_t)wib * mpad * ts;
    const int grp = lane >> 2, tig = lane & 3;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t q = first + gw; q < first + count; q += nw) {
        int8_transpose_to_smem(pop + (size_t)q * m * m, m, mpad, kpad, ts, T, lane);
        uint32_t acc = 0;
        for (int i0 = 0; i0 < mpad; i0 += 16) {
            // only column tiles that reach above the diagonal of this row tile
            for (int j0 = i0 & ~7; j0 < mpad; j0 += 8) {
                float d[4] = {0.f, 0.f, 0.f, 0.f};
                for (int k0 = 0; k0 < kpad; k0 += 32) {
                    uint32_t a[4], b[2];
                    const int8_t *ta = T + (i0 + grp) * ts + k0 + tig * 4;
                    a[0] = i8_to_e4m3_z(*reinterpret_cast<const uint32_t *>(ta));
                    a[1] = i8_to_e4m3_z(*reinterpret_cast<const uint32_t *>(ta + 8 * ts));
                    a[2] = i8_to_e4m3_z(*reinterpret_cast<const uint32_t *>(ta + 16));
                    a[3] = i8_to_e4m3_z(*reinterpret_cast<const uint32_t *>(ta + 8 * ts + 16));
                    const int8_t *tb = T + (j0 + grp) * ts + k0 + tig * 4;
                    b[0] = i8_to_e4m3_z(*reinterpret_cast<const uint32_t *>(tb));
                    b[1] = i8_to_e4m3_z(*reinterpret_cast<const uint32_t *>(tb + 16));
                    mma_e4m3_16832(d, a, b);
                }
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int i = i0 + grp + ((e >> 1) << 3);
                    const int j = j0 + tig * 2 + (e & 1);
                    if (i < j && j < m)
                        acc += fit_term<KIND>(gram_value(d[e]));
                }
            }
        }
        const uint32_t f = fit_finish<KIND>(warp_sum(acc));
        if (lane == 0)
            fit[q] = f;
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// F_sq through the row Gram.  For any +-1 matrix, the sum over i < j of the
// squared column inner products equals the sum over r < s of the squared row
// inner products (both are (||Q^T Q||_F^2 - m^3) / 2, since the diagonals are
// m and ||Q^T Q||_F = ||Q Q^T||_F).  R = Q Q^T maps onto mma.sync row.col
// with both operands read straight from the row-major int8 matrix: A holds
// rows r, B holds rows s, k runs along a row.  The sum over k is the same
// under any consistent relabelling of k, so every lane reads 8 contiguous
// bytes of a row per 32-wide k step (k slots 4t..4t+3 <- bytes 8t..8t+3 and
// k slots 16+4t..19+4t <- bytes 8t+4..8t+7) and a warp's loads are
// fully coalesced.
// ---------------------------------------------------------------------------

// Sum over the upper-triangle entries of one 16 x 8 accumulator tile of the
// row Gram: d^2 in FP32, exact while a lane's sum stays below 2^24 (at most
// 4 * tiles_per_lane * m^2 = 4 * 34 * 65536 < 2^24 for m <= 256).  Only the
// two tiles on the diagonal (cj = 2 ri, 2 ri + 1) need the entry mask.
__device__ __forceinline__ float tile_sq_sum(const float (&d)[4], int ri, int cj, int grp, int tig, float acc)
{
    if (cj >= 2 * ri + 2) {
#pragma unroll
        for (int e = 0; e < 4; ++e)
            acc = fmaf(d[e], d[e], acc);
    } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int r = 16 * ri + grp + ((e >> 1) << 3);
            const int c = 8 * cj + tig * 2 + (e & 1);
            acc = fmaf(c > r ? d[e] : 0.f, d[e], acc);
        }
    }
    return acc;
}

// m in {32, 64}: one warp per matrix, the whole matrix in registers
// (lane (g, t) holds rows g + 8q, q < m/8, bytes 8t..8t+7 of every 32-byte
// k step).
template <int M, bool E4M3>
__global__ void __launch_bounds__(256) k_fsq_imma_regs(const int8_t *__restrict__ pop, int64_t first, int64_t count,
                                                      uint32_t *__restrict__ fit)
{
    constexpr int RG = M / 8, KS = M / 32, MT = M / 16;
    const int lane = threadIdx.x & 31, grp = lane >> 2, tig = lane & 3;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    uint2 cur[RG][KS], nxt[RG][KS];
    auto load = [&](int64_t q, uint2 (&f)[RG][KS]) {
        const uint8_t *Q = reinterpret_cast<const uint8_t *>(pop) + (size_t)q * M * M;
#pragma unroll
        for (int r = 0; r < RG; ++r)
#pragma unroll
            for (int ks = 0; ks < KS; ++ks)
                f[r][ks] = __ldg(reinterpret_cast<const uint2 *>(Q + (size_t)(grp + 8 * r) * M + ks * 32 + tig * 8));
    };
    int64_t q = first + gw;
    if (q < first + count)
        load(q, cur);
    for (; q < first + count; q += nw) {
        const int64_t qn = q + nw;
        if (qn < first + count)
            load(qn, nxt);
        float acc = 0.f;  // exact: at most 4 * 20 entries of m^2 = 4096 per lane
#pragma unroll
        for (int ri = 0; ri < MT; ++ri) {
#pragma unroll
            for (int cj = 2 * ri; cj < RG; ++cj) {
                float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int ks = 0; ks < KS; ++ks) {
                    const uint32_t a[4] = {fp8_operand<E4M3>(cur[2 * ri][ks].x), fp8_operand<E4M3>(cur[2 * ri + 1][ks].x),
                                           fp8_operand<E4M3>(cur[2 * ri][ks].y), fp8_operand<E4M3>(cur[2 * ri + 1][ks].y)};
                    const uint32_t b[2] = {fp8_operand<E4M3>(cur[cj][ks].x), fp8_operand<E4M3>(cur[cj][ks].y)};
                    mma_e4m3_16832(d, a, b);
                }
                acc = tile_sq_sum(d, ri, cj, grp, tig, acc);
            }
        }
        const uint32_t f = warp_sum((uint32_t)acc);
        if (lane == 0)
            fit[q] = f;
#pragma unroll
        for (int r = 0; r < RG; ++r)
#pragma unroll
            for (int ks = 0; ks < KS; ++ks)
                cur[r][ks] = nxt[r][ks];
    }
}

// m a multiple of 32 above 64: one block of 4 warps per matrix, the matrix
// staged in shared memory with rows padded by 32 bytes (a half-warp's 8-byte
// reads of 4 rows then cover all 32 banks), the upper-triangle 16 x 8 tiles
// of R dealt round-robin to the warps.
constexpr int kMmaSmemThreads = 256;  // 8 warps per block

// m in {96, 128, ..., 256} (multiple of 32): one matrix per block at a time,
// staged in shared memory with padded rows (stride m + 32 bytes); two
// buffers, the next matrix's rows arriving by cp.async while the current
// one is multiplied.  Each warp takes a contiguous range of the upper tiles
// (16 rows x 8 rows of the row Gram) in row-block order and keeps the A
// fragments of a row block in registers across its tiles: one shared-memory
// operand load per MMA.
template <int M, bool E4M3>
__global__ void __launch_bounds__(kMmaSmemThreads) k_fsq_imma_smem(const int8_t *__restrict__ pop, int64_t first,
                                                                  int64_t count, uint32_t *__restrict__ fit)
{
    extern __shared__ __align__(16) uint8_t s_q[];
    __shared__ uint32_t s_part[kMmaSmemThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, grp = lane >> 2, tig = lane & 3;
    constexpr int NW = kMmaSmemThreads / 32;
    constexpr int RS = M + 32;  // padded row stride in bytes
    constexpr int KS = M / 32, MT = M / 16, CT = M / 8;
    constexpr int T = MT * CT - MT * (MT - 1);  // upper tiles
    constexpr size_t BSZ = (size_t)M * RS;
    constexpr int CHUNKS = M * M / 16, PER_ROW = M / 16;
    auto issue = [&](int64_t q, int b) {
        const uint4 *src = reinterpret_cast<const uint4 *>(pop + (size_t)q * M * M);
        uint8_t *dst = s_q + (size_t)b * BSZ;
        for (int c = threadIdx.x; c < CHUNKS; c += blockDim.x)
            cp_async16(dst + (c / PER_ROW) * RS + (c % PER_ROW) * 16, src + c);
        cp_async_commit();
    };
    // this warp's tiles [t0, t1) and the (ri, cj) of t0
    const int t0 = warp * T / NW, t1 = (warp + 1) * T / NW;
    int ri0 = 0, before = 0;
    while (before + (CT - 2 * ri0) <= t0) {
        before += CT - 2 * ri0;
        ++ri0;
    }
    const int cj0 = 2 * ri0 + (t0 - before);
    const int64_t end = first + count;
    int64_t q = first + blockIdx.x;
    int buf = 0;
    if (q < end)
        issue(q, buf);
    for (; q < end; q += gridDim.x) {
        const int64_t qn = q + gridDim.x;
        if (qn < end) {
            issue(qn, buf ^ 1);
            cp_async_wait_group<1>();
        } else {
            cp_async_wait_group<0>();
        }
        __syncthreads();
        const uint8_t *Q = s_q + (size_t)buf * BSZ + grp * RS + tig * 8;
        float acc = 0.f;
        uint32_t a[KS][4];
        int ri = ri0, cj = cj0, a_ri = -1;
        for (int t = t0; t < t1; ++t) {
            if (a_ri != ri) {
                const uint8_t *qa = Q + 16 * ri * RS;
#pragma unroll
                for (int ks = 0; ks < KS; ++ks) {
                    const uint2 a0 = *reinterpret_cast<const uint2 *>(qa + ks * 32);
                    const uint2 a1 = *reinterpret_cast<const uint2 *>(qa + 8 * RS + ks * 32);
                    a[ks][0] = fp8_operand<E4M3>(a0.x);
                    a[ks][1] = fp8_operand<E4M3>(a1.x);
                    a[ks][2] = fp8_operand<E4M3>(a0.y);
                    a[ks][3] = fp8_operand<E4M3>(a1.y);
                }
                a_ri = ri;
            }
            float d[4] = {0.f, 0.f, 0.f, 0.f};
            const uint8_t *qb = Q + 8 * cj * RS;
#pragma unroll
            for (int ks = 0; ks < KS; ++ks) {
                const uint2 b0 = *reinterpret_cast<const uint2 *>(qb + ks * 32);
                const uint32_t b[2] = {fp8_operand<E4M3>(b0.x), fp8_operand<E4M3>(b0.y)};
                mma_e4m3_16832(d, a[ks], b);
            }
            acc = tile_sq_sum(d, ri, cj, grp, tig, acc);
            if (++cj == CT) {
                ++ri;
                cj = 2 * ri;
            }
        }
        // the lane sum is an exact integer below 2^24; reduce in integers
        const uint32_t wsum = warp_sum((uint32_t)acc);
        if (lane == 0)
            s_part[warp] = wsum;
        __syncthreads();  // also: every warp is done with `buf` before it is refilled
        if (threadIdx.x == 0) {
            uint32_t f = 0;
            for (int w = 0; w < NW; ++w)
                f += s_part[w];
            fit[q] = f;
        }
        buf ^= 1;
    }
}

// F_sq with CUDA-core 4-way byte dot products on the row Gram: one warp per
// matrix staged in shared memory; lane r owns rows r, r + 32, ... and pairs
// each with the rows that follow it (mod m) by the same circular rule as
// the popcount kernels.
__global__ void __launch_bounds__(128) k_fsq_dp4a_rows(const int8_t *__restrict__ pop, int m, int64_t first,
                                                       int64_t count, uint32_t *__restrict__ fit)
{
    extern __shared__ __align__(16) uint8_t s_rows[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int rsw = m / 4 + 1;  // padded row stride in words (odd: conflict-free column reads)
    uint32_t *R = reinterpret_cast<uint32_t *>(s_rows) + (size_t)wib * m * rsw;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int kw = m / 4, half = m >> 1;
    for (int64_t q = first + gw; q < first + count; q += nw) {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(pop + (size_t)q * m * m);
        for (int e = lane; e < m * kw; e += 32)
            R[(e / kw) * rsw + (e % kw)] = __ldg(src + e);
        __syncwarp();
        uint32_t acc = 0;
        for (int a = lane; a < m; a += 32) {
            const uint32_t *ra = R + a * rsw;
            const int smax = a < half ? half : half - 1;
            int b = a;
            for (int s = 1; s <= smax; ++s) {
                b = (b + 1 == m) ? 0 : b + 1;
                const uint32_t *rb = R + b * rsw;
                int g = 0;
                for (int k = 0; k < kw; ++k)
                    g = __dp4a((int)ra[k], (int)rb[k], g);
                acc += (uint32_t)(g * g);
            }
        }
        acc = warp_sum(acc);
        if (lane == 0)
            fit[q] = acc;
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Dispatch
// ---------------------------------------------------------------------------
bool fitness_path_supported(int storage, int m, int path)
{
    if (path == 5)
        return storage == ST_BITS || storage == ST_INT8;
    if (path == 1 || path == 2)
        return storage == ST_INT8;
    if (path == 6)
        return storage == ST_E4M3;
    return false;
}

static int grid_for_warps(int64_t count, int warps_per_block)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (count + warps_per_block - 1) / warps_per_block;
    const int64_t cap = (int64_t)(sms > 0 ? sms : 148) * 64;
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

template <int M, bool E4M3>
static void launch_fsq_mma_smem(const int8_t *pop, int64_t first, int64_t count, uint32_t *fit, size_t smem, int sms,
                                cudaStream_t s)
{
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_fsq_imma_smem<M, E4M3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    // as many resident blocks as shared memory allows, each looping over matrices
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fsq_imma_smem<M, E4M3>, kMmaSmemThreads, smem);
    const int64_t cap = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
    const int64_t want = count < cap ? count : cap;
    k_fsq_imma_smem<M, E4M3><<<(unsigned)(want > 0 ? want : 1), kMmaSmemThreads, smem, s>>>(pop, first, count, fit);
}

template <int KIND>
static cudaError_t fitness_kind(const void *pop, int storage, int m, int64_t first, int64_t count, int path,
                                uint32_t *fit, cudaStream_t s)
{
    const int W = words_per_col(m);
    if (path == 5 && storage == ST_BITS && m <= 32) {
        const int bs = 128;
        const unsigned grid = (unsigned)((count + bs - 1) / bs);
        const uint32_t *p = (const uint32_t *)pop;
        switch (m) {
#define HADGA_FT(M)                                                                                         \
    case M:                                                                                                 \
        k_fit_bits_thread<M, KIND><<<grid, bs, 0, s>>>(p, first, count, fit);                               \
        break;
            HADGA_FT(4) HADGA_FT(8) HADGA_FT(12) HADGA_FT(16) HADGA_FT(20) HADGA_FT(24) HADGA_FT(28) HADGA_FT(32)
#undef HADGA_FT
        default:
            return cudaErrorInvalidValue;
        }
        note_launches(1);
        return cudaGetLastError();
    }
    if (path == 5) {
        const int wpb = 8;
        const size_t smem = (size_t)wpb * col_set_words(m, W) * 4;  // at most 64 KiB (m = 256)
        const int grid = grid_for_warps(count, wpb);
        switch (W) {
#define HADGA_FW(WW)                                                                                        \
    case WW:                                                                                                \
        if (storage == ST_BITS) {                                                                           \
            cudaFuncSetAttribute(k_fit_bits_warp<WW, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                                 (int)smem);                                                                \
            k_fit_bits_warp<WW, KIND><<<grid, wpb * 32, smem, s>>>((const uint32_t *)pop, m, first, count,  \
                                                                  fit);                                     \
        } else {                                                                                            \
            cudaFuncSetAttribute(k_fit_int8_popc<WW, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                                 (int)smem);                                                                \
            k_fit_int8_popc<WW, KIND><<<grid, wpb * 32, smem, s>>>((const int8_t *)pop, m, first, count,    \
                                                                  fit);                                     \
        }                                                                                                   \
        break;
            HADGA_FW(1) HADGA_FW(2) HADGA_FW(3) HADGA_FW(4) HADGA_FW(5) HADGA_FW(6) HADGA_FW(7) HADGA_FW(8)
#undef HADGA_FW
        default:
            return cudaErrorInvalidValue;
        }
        note_launches(1);
        return cudaGetLastError();
    }
    // F_sq on int8: row-Gram kernels (no transpose)
    // paths 2 (int8 storage) and 6 (e4m3 storage): warp-level FP8 MMA
    const bool fp8 = path == 6;
    if (KIND == FIT_SQ && (path == 2 || path == 6) && (m == 32 || m == 64)) {
        const int grid = grid_for_warps(count, 8);
        const int8_t *q = (const int8_t *)pop;
        if (m == 32)
            fp8 ? k_fsq_imma_regs<32, true><<<grid, 256, 0, s>>>(q, first, count, fit)
                : k_fsq_imma_regs<32, false><<<grid, 256, 0, s>>>(q, first, count, fit);
        else
            fp8 ? k_fsq_imma_regs<64, true><<<grid, 256, 0, s>>>(q, first, count, fit)
                : k_fsq_imma_regs<64, false><<<grid, 256, 0, s>>>(q, first, count, fit);
        note_launches(1);
        return cudaGetLastError();
    }
    if (KIND == FIT_SQ && (path == 2 || path == 6) && m % 32 == 0) {
        const size_t smem = 2 * (size_t)m * (m + 32);  // two staging buffers
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int8_t *q = (const int8_t *)pop;
        switch (m) {
#define HADGA_MS(MM)                                                                                         \
    case MM:                                                                                                 \
        if (fp8)                                                                                             \
            launch_fsq_mma_smem<MM, true>(q, first, count, fit, smem, sms, s);                               \
        else                                                                                                 \
            launch_fsq_mma_smem<MM, false>(q, first, count, fit, smem, sms, s);                              \
        break;
            HADGA_MS(96) HADGA_MS(128) HADGA_MS(160) HADGA_MS(192) HADGA_MS(224) HADGA_MS(256)
#undef HADGA_MS
        default:
            return cudaErrorInvalidValue;
        }
        note_launches(1);
        return cudaGetLastError();
    }
    if (KIND == FIT_SQ && path == 1) {
        const size_t per_warp = (size_t)m * (m / 4 + 1) * 4;
        int wpb = 4;
        while (wpb > 1 && per_warp * wpb > 200 * 1024)
            --wpb;
        const size_t smem = (size_t)wpb * per_warp;
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k_fsq_dp4a_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        const int grid = grid_for_warps(count, wpb);
        k_fsq_dp4a_rows<<<grid, wpb * 32, smem, s>>>((const int8_t *)pop, m, first, count, fit);
        note_launches(1);
        return cudaGetLastError();
    }
    // INT32 / IMMA on int8, column Gram on a transposed copy
    const int kpad = (m + 31) & ~31, mpad = (m + 15) & ~15, ts = kpad + 16;
    const size_t per_warp = (size_t)mpad * ts;
    int wpb = 4;
    while (wpb > 1 && per_warp * wpb > 96 * 1024)
        wpb >>= 1;
    const size_t smem = per_warp * wpb;
    const int grid = grid_for_warps(count, wpb);
    if (path == 1) {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k_fit_int8_dp4a<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_fit_int8_dp4a<KIND><<<grid, wpb * 32, smem, s>>>((const int8_t *)pop, m, first, count, fit);
    } else {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k_fit_int8_imma<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_fit_int8_imma<KIND><<<grid, wpb * 32, smem, s>>>((const int8_t *)pop, m, first, count, fit);
    }
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_fitness(const void *pop, int storage, int m, int64_t first, int64_t count, int kind, int path,
                           uint32_t *fit, cudaStream_t s)
{
    if (count <= 0)
        return cudaSuccess;
    switch (kind) {
    case FIT_SQ: return fitness_kind<FIT_SQ>(pop, storage, m, first, count, path, fit, s);
    case FIT_ABS: return fitness_kind<FIT_ABS>(pop, storage, m, first, count, path, fit, s);
    case FIT_NNZ: return fitness_kind<FIT_NNZ>(pop, storage, m, first, count, path, fit, s);
    default: return cudaErrorInvalidValue;
    }
}

} // namespace hadga
