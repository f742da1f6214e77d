// k_tc.cu -- batched Gram + F_sq on the 5th-generation tensor cores
// (tcgen05) for populations stored as FP8 e4m3 or BF16 (+-1 exactly
// representable; FP32 accumulation of at most 256 products of +-1 is exact).
//
// F_sq is taken from the row Gram R = Q Q^T (for +-1 matrices the sum of
// squared off-diagonal entries above the diagonal equals the column Gram's),
// so both MMA operands are the row-major matrix itself, K-major, as the TMA
// copy lands it.  A job is a tile of 128 consecutive rows of the population
// (128/m whole matrices for m <= 128; for m = 256 a job is one matrix, 256
// rows, two M-tiles of which only the upper-triangle blocks are computed).
// The K extent of a row is cut into chunks of 128 bytes (or the row, if
// shorter); each chunk is one pipeline stage, copied by TMA with the matching
// 32/64/128-byte swizzle.
//
// Roles (warp specialised, one block per SM):
//   warp 0   one thread issues the TMA copies into a ring of stages (up to
//            32 stages of rows x chunk bytes within 160 KiB)
//   warp 1   allocates all 512 TMEM columns; one thread issues tcgen05.mma
//            per stage and commits to the stage's "empty" barrier; at the end
//            of a job it commits to the accumulator's "full" barrier (four
//            128-column accumulators for m <= 128, one 384-column pair of
//            blocks for m = 256).  Ring positions and phases are counters
//            (no division in the issue loop).
//   warp 10  with four accumulators (m <= 128), a second MMA issuer: warp 1
//            takes the block's even jobs, warp 10 the odd ones.  The stage
//            ring is then split in two halves, one per issuer: the producer
//            fills half r for the jobs of issuer r only, so every use of a
//            stage follows a use by the same issuer and a parity wait on its
//            "full" barrier can never pass on the phase of an earlier lap
//            that the other issuer has not consumed yet
//   warps 2-9  two epilogue groups of four warps, taking alternate jobs with
//            four accumulators, or both on every job at m = 256 (group 0
//            reads columns 0..191, group 1 columns 192..383, so the single
//            accumulator is free again after half the reads): wait for the
//            accumulator, read it with tcgen05.ld (warp w reads TMEM lanes
//            32(w%4)..32(w%4)+31 = tile rows), free it, then square, sum and
//            write the fitness
// Every mbarrier wait is bounded (about two seconds); on a timeout the block
// records ERR_TIMEOUT, drains its outstanding copies with bounded waits,
// frees its TMEM and returns.
#include <cuda.h>

#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"

namespace hadga {

namespace {

constexpr int kTcThreads = 352;  // 11 warps: producer, MMA, two epilogue groups of four, second MMA
constexpr int kTcMma2Warp = 10;  // the second MMA issuer
constexpr int kMaxStages = 32;
constexpr uint32_t kRingBytes = 160 * 1024;  // shared memory of the stage ring

// Error word of launches that come without one (the stateless batch call).
__device__ uint32_t g_tc_err;

struct TcParams {
    int64_t P;          // matrices
    int32_t m;          // order (32, 64, 128, 256)
    int32_t esize;      // bytes per element (1 e4m3, 2 bf16)
    int32_t kb;         // chunk width in bytes (<= 128)
    int32_t nchunks;    // chunks per row
    int32_t rows;       // rows per job (128, or 256 for m = 256)
    int32_t nstages;    // stages in the ring (each rows x kb bytes)
    int64_t jobs;
    uint32_t idesc_n128, idesc_n256;  // instruction descriptors
    uint32_t layout;    // smem descriptor layout type of the swizzle
    uint32_t *fit;
    uint32_t *err;
};

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int32_t x, int32_t y, uint64_t *bar)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
                 "[%4];" ::"r"(smem_u32(dst)),
                 "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
                 : "memory");
}

// Shared-memory matrix descriptor of a K-major swizzled operand: start
// address, leading byte offset (unused for swizzled K-major, 1), stride byte
// offset between groups of 8 rows, descriptor version 1, layout type.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t sbo, uint32_t layout)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)1u << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1u << 46;
    d |= (uint64_t)layout << 61;
    return d;
}

template <bool BF16>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc)
{
    if (BF16)
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
                     "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
    else
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
                     "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 consecutive fp32 accumulator columns of this thread's TMEM lane, without
// waiting (tmem_wait_ld completes every load issued so far).
__device__ __forceinline__ void tmem_ld32_nowait(uint32_t taddr, uint32_t (&v)[32])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                   "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                   "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                   "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                 : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Sum of squares of U x 32 consecutive accumulator columns of this thread's
// lane (exact: integer values, partial sums <= 2^24), four independent chains.
template <int U>
__device__ __forceinline__ float sq_cols(uint32_t taddr)
{
    uint32_t v[U][32];
#pragma unroll
    for (int u = 0; u < U; ++u)
        tmem_ld32_nowait(taddr + (uint32_t)(u * 32), v[u]);
    tmem_wait_ld();
    float s[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
        for (int c = 0; c < 32; ++c) {
            const float x = __uint_as_float(v[u][c]);
            s[c & 3] = fmaf(x, x, s[c & 3]);
        }
    return (s[0] + s[1]) + (s[2] + s[3]);
}

} // namespace

// SPLIT: m <= 128, two MMA issuers, each with its own half of the stage ring
// (four accumulators); otherwise m = 256, one issuer on the whole ring and one
// accumulator. The two are separate instantiations so that neither carries the
// other's loops or epilogue.
template <bool BF16, bool SPLIT>
__global__ void __launch_bounds__(kTcThreads, 1) k_fsq_tc(const __grid_constant__ CUtensorMap map,
                                                          const __grid_constant__ TcParams prm)
{
    extern __shared__ __align__(1024) uint8_t dyn_raw[];
    // 1024-byte alignment keeps every stage on the swizzle pattern's base
    uint8_t *stages = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(dyn_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t full[kMaxStages], empty[kMaxStages], acc_full[4], acc_empty[4], drain[2];
    __shared__ uint32_t tmem_base;
    // partial sums of the matrices of a job: [accumulator][matrix of the tile][use parity]
    __shared__ unsigned long long part_sum[4][2][2];
    __shared__ uint32_t part_cnt[4][2][2];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m = prm.m, rows = prm.rows, nch = prm.nchunks, kb = prm.kb, S = prm.nstages;
    const uint32_t sbytes = (uint32_t)rows * (uint32_t)kb;  // bytes of one stage
    constexpr int nacc = SPLIT ? 4 : 1;
    // epilogue groups: with four accumulators (m <= 128) they take alternate
    // jobs; at m = 256 both read every job, each half of its 384 columns
    constexpr int ngroups = 2;
    const uint32_t tmem_cols = 512u;
    uint32_t *err = prm.err ? prm.err : &g_tc_err;

    if (threadIdx.x == 0) {
        for (int st = 0; st < S; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], 1);
        }
        for (int b = 0; b < 4; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], SPLIT ? 128 : 256);
            for (int g = 0; g < 2; ++g)
                for (int u = 0; u < 2; ++u) {
                    part_sum[b][g][u] = 0ull;
                    part_cnt[b][g][u] = 0u;
                }
        }
        mbar_init(&drain[0], 1);
        mbar_init(&drain[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tbase = tmem_base;

    // MMA issuers and the stage ring halves they own (one ring of S stages
    // with a single issuer; two halves of SR stages with two)
    constexpr int nis = SPLIT ? 2 : 1;
    const int SR = S / nis;
    if (warp == 0) {
        // ---- TMA producer ----------------------------------------------------
        if (!SPLIT && lane == 0) {
            // one issuer, one ring (m = 256)
            uint32_t it = 0;
            int issued = 0;
            int st = 0;         // stage of copy `it`
            uint32_t sph = 0u;  // parity of that stage's current use
            bool ok = true;
            for (int64_t j = blockIdx.x; j < prm.jobs && ok; j += gridDim.x) {
                for (int c = 0; c < nch; ++c, ++it) {
                    if (!mbar_wait(&empty[st], sph ^ 1u, err)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&full[st], sbytes);
                    const int32_t x = c * (kb / prm.esize);
                    for (int h = 0; h < rows / 128; ++h)
                        tma_load_2d(stages + (size_t)st * sbytes + (size_t)h * 128 * kb, &map, x,
                                    (int32_t)(j * rows + h * 128), &full[st]);
                    issued = issued < S ? issued + 1 : S;
                    if (++st == S) {
                        st = 0;
                        sph ^= 1u;
                    }
                }
            }
            if (!ok) {
                // drain: let copies already in flight land before the block exits
                for (int q = 0; q < issued; ++q) {
                    const uint32_t itq = it - 1u - (uint32_t)q;
                    mbar_wait(&full[itq % (uint32_t)S], (itq / (uint32_t)S) & 1u, err);
                }
            }
        } else if (SPLIT && lane == 0) {
            // two issuers, two ring halves (m <= 128)
            // per ring half (issuer) 0 / 1, kept in registers: next stage
            // (relative), parity of its current use, uses issued so far
            int pos0 = 0, pos1 = 0;
            uint32_t sph0 = 0u, sph1 = 0u, used0 = 0u, used1 = 0u;
            int who = 0;  // issuer (ring half) of the next job
            bool ok = true;
            for (int64_t j = blockIdx.x; j < prm.jobs && ok; j += gridDim.x) {
                const bool second = who == 1;
                if (++who == nis)
                    who = 0;
                int pos = second ? pos1 : pos0;
                uint32_t sph = second ? sph1 : sph0;
                const int s0 = second ? SR : 0;
                int issued = 0;
                for (int c = 0; c < nch; ++c) {
                    const int st = s0 + pos;
                    if (!mbar_wait(&empty[st], sph ^ 1u, err)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&full[st], sbytes);
                    const int32_t x = c * (kb / prm.esize);
                    for (int h = 0; h < rows / 128; ++h)
                        tma_load_2d(stages + (size_t)st * sbytes + (size_t)h * 128 * kb, &map, x,
                                    (int32_t)(j * rows + h * 128), &full[st]);
                    ++issued;
                    if (++pos == SR) {
                        pos = 0;
                        sph ^= 1u;
                    }
                }
                if (second) {
                    pos1 = pos;
                    sph1 = sph;
                    used1 += (uint32_t)issued;
                } else {
                    pos0 = pos;
                    sph0 = sph;
                    used0 += (uint32_t)issued;
                }
            }
            if (!ok) {
                // drain: let copies already in flight land before the block exits
                // (the last min(used, SR) uses of each half)
                for (int r = 0; r < nis; ++r) {
                    const uint32_t used = r ? used1 : used0;
                    const uint32_t n = used < (uint32_t)SR ? used : (uint32_t)SR;
                    for (uint32_t q = 0; q < n; ++q) {
                        const uint32_t u = used - 1u - q;
                        mbar_wait(&full[r * SR + (int)(u % (uint32_t)SR)], (u / (uint32_t)SR) & 1u, err);
                    }
                }
            }
        }
    } else if (warp == 1 || warp == kTcMma2Warp) {
        // ---- MMA issuers ----------------------------------------------------------
        // With several accumulators (m <= 128) warp 1 issues the block's even jobs
        // and warp kTcMma2Warp the odd ones, each on its own accumulators and its
        // own half of the stage ring (the issue of a 128 x 128 job's MMAs and
        // commits, not the tensor pipe, paces one thread); m = 256 has one
        // accumulator and one issuer.
        const int me = warp == 1 ? 0 : 1;
        // TWO: compiled with the job split (the single-issuer loop keeps none of it)
        auto issue = [&](auto two) {
            constexpr bool TWO = decltype(two)::value;
            const uint32_t sbo = 8u * (uint32_t)kb;
            // ring positions kept as counters: no division in the issue loop
            // first stage and length of this issuer's ring (half of the ring with two issuers)
            const int s0 = TWO ? me * SR : 0, sr = TWO ? SR : S;
            int st = s0, b = 0, who = 0;
            uint32_t sph = 0u, aph = 0u;  // parities of the stage's and accumulator's current use
            bool ok = true;
            for (int64_t j = blockIdx.x; j < prm.jobs && ok; j += gridDim.x) {
                const bool mine = !TWO || who == me;
                if (TWO && ++who == 2)
                    who = 0;
                if (!mine) {
                    // the other issuer's job: its stages are in the other half; only
                    // the accumulator use advances
                    if (++b == nacc) {
                        b = 0;
                        aph ^= 1u;
                    }
                    continue;
                }
                if (!mbar_wait(&acc_empty[b], aph ^ 1u, err)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d0 = tbase + (uint32_t)b * 128u;
                for (int c = 0; c < nch; ++c) {
                    if (!mbar_wait(&full[st], sph, err)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t base = smem_u32(stages + (size_t)st * sbytes);
                    for (int ks = 0; ks < kb / 32; ++ks) {
                        const uint32_t acc = (c > 0 || ks > 0) ? 1u : 0u;
                        const uint32_t koff = (uint32_t)ks * 32u;
                        if constexpr (!SPLIT) {
                            // m = 256, upper blocks: rows 0..127 x cols 0..255, rows 128..255 x cols 128..255
                            const uint64_t a0 = smem_desc(base + koff, sbo, prm.layout);
                            const uint64_t a1 = smem_desc(base + 128u * (uint32_t)kb + koff, sbo, prm.layout);
                            mma<BF16>(tbase, a0, a0, prm.idesc_n256, acc);
                            mma<BF16>(tbase + 256u, a1, a1, prm.idesc_n128, acc);
                        } else {
                            const uint64_t a = smem_desc(base + koff, sbo, prm.layout);
                            mma<BF16>(d0, a, a, prm.idesc_n128, acc);
                        }
                    }
                    mma_commit(&empty[st]);  // the stage is free once these MMAs have read it
                    if (++st == s0 + sr) {
                        st = s0;
                        sph ^= 1u;
                    }
                }
                if (!ok)
                    break;
                mma_commit(&acc_full[b]);  // the accumulator is complete
                if (++b == nacc) {
                    b = 0;
                    aph ^= 1u;
                }
            }
            if (!ok) {
                // make sure none of this thread's MMAs is still writing TMEM before it is freed
                mma_commit(&drain[me]);
                mbar_wait(&drain[me], 0u, err);
            }
        };
        if (lane == 0 && me < nis) {
            if constexpr (SPLIT)
                issue(std::true_type{});
            else
                issue(std::false_type{});
        }
    } else {
        // ---- epilogue: warps 2..5 (group 0) and 6..9 (group 1) --------------------
        // Sum over r < s of R_rs^2 = (sum over all r, s of R_rs^2 - m^3) / 2 (the
        // diagonal is m): each thread squares and adds every accumulator of its row
        // block with one FFMA per entry; partial sums stay integers <= 2^24, exact.
        const int grp = (warp - 2) >> 2;      // epilogue group
        const int q = warp & 3;               // TMEM sub-partition this warp may read
        const int t = q * 32 + lane;          // tile row (and TMEM lane)
        if (grp < ngroups) {
            // the block's jobs in order: group gsel takes the job, on accumulator
            // bn whose use has parity aph (counters, no division)
            int gsel = 0, bn = 0;
            uint32_t aph = 0u;
            for (int64_t j = blockIdx.x; j < prm.jobs; j += gridDim.x) {
                const bool mine = !SPLIT || gsel == grp;
                const int b = bn;
                const uint32_t ph = aph;
                if (++gsel == ngroups)
                    gsel = 0;
                if (++bn == nacc) {
                    bn = 0;
                    aph ^= 1u;
                }
                if (!mine)
                    continue;
                if (!mbar_wait(&acc_full[b], ph, err))
                    break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t lane_addr = tbase + ((uint32_t)(q * 32) << 16);
                float sum_a = 0.f, sum_b = 0.f;
                if constexpr (!SPLIT) {
                    // m = 256: row t of the first block: columns 0..127 count once, 128..255 twice
                    // (their mirror images below the diagonal are not computed); row
                    // 128 + t of the second block: its 128 columns once.  Group 0 reads
                    // columns 0..191, group 1 columns 192..383.
                    if (grp == 0) {
                        sum_a = sq_cols<4>(lane_addr);
                        sum_b = sq_cols<2>(lane_addr + 128u);
                    } else {
                        sum_b = sq_cols<2>(lane_addr + 192u);
                        sum_a = sq_cols<4>(lane_addr + 256u);
                    }
                } else {
                    const int g = t / m;
                    const uint32_t col0 = lane_addr + (uint32_t)b * 128u + (uint32_t)(g * m);
                    sum_a = m == 32 ? sq_cols<1>(col0) : m == 64 ? sq_cols<2>(col0) : sq_cols<4>(col0);
                }
                // the accumulator is read (tcgen05.wait::ld inside sq_cols): hand it
                // back to the MMA issuer before the reduction
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                mbar_arrive(&acc_empty[b]);
                const int use = (int)ph;
                unsigned long long tot = (unsigned long long)(uint32_t)sum_a + 2ull * (uint32_t)sum_b;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
                    tot += __shfl_xor_sync(0xFFFFFFFFu, tot, o);
                const unsigned long long m3 = (unsigned long long)m * m * m;
                if (SPLIT && m <= 32) {
                    // one warp per matrix
                    const int64_t mat = (j * rows + (int64_t)q * 32) / m;
                    if (lane == 0 && mat < prm.P)
                        prm.fit[mat] = (uint32_t)((tot - m3) >> 1);
                } else if (lane == 0) {
                    // m = 64: warps of sub-partitions 2g, 2g+1 hold matrix g; m = 128: all
                    // four of the group; m = 256: all eight of both groups
                    const int g = (m == 64) ? (q >> 1) : 0;
                    const uint32_t need = !SPLIT ? 8u : (m == 64) ? 2u : 4u;
                    atomicAdd(&part_sum[b][g][use], tot);
                    __threadfence_block();
                    if (atomicAdd(&part_cnt[b][g][use], 1u) + 1u == need) {
                        const unsigned long long all = atomicExch(&part_sum[b][g][use], 0ull);
                        part_cnt[b][g][use] = 0u;
                        const int64_t mat = (j * rows) / m + g;
                        if (mat < prm.P)
                            prm.fit[mat] = (uint32_t)((all - m3) >> 1);
                    }
                }
                // The combining slot of use parity u is taken again by the job two
                // uses later on this accumulator, whose MMA waits for every thread
                // reading the accumulator (the group, or both groups at m = 256) to
                // have read the use in between, i.e. to have finished this job's
                // combination first.
                __syncwarp();
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(tmem_cols)
                     : "memory");
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

uint32_t idesc(bool bf16, int n)
{
    uint32_t d = 0;
    d |= 1u << 4;                          // accumulator F32
    if (bf16)
        d |= (1u << 7) | (1u << 10);       // A, B BF16 (kind::f16); E4M3 is 0 (kind::f8f6f4)
    d |= (uint32_t)(n >> 3) << 17;         // N / 8
    d |= (uint32_t)(128 >> 4) << 24;       // M / 16
    return d;                              // both operands K-major, dense, no negation
}

} // namespace

bool fitness_tc_supported(int storage, int m)
{
    return (storage == ST_E4M3 || storage == ST_BF16) && (m == 32 || m == 64 || m == 128 || m == 256) &&
           encode_fn() != nullptr;
}

cudaError_t launch_fitness_tc(const void *pop, int storage, int m, int64_t first, int64_t count, int kind,
                              uint32_t *fit, uint32_t *err, cudaStream_t s)
{
    if (kind != FIT_SQ || !fitness_tc_supported(storage, m))
        return cudaErrorNotSupported;
    if (count <= 0)
        return cudaSuccess;
    const bool bf16 = storage == ST_BF16;
    const int esize = bf16 ? 2 : 1;
    const int row_bytes = m * esize;
    TcParams prm{};
    prm.P = count;
    prm.m = m;
    prm.esize = esize;
    prm.kb = row_bytes < 128 ? row_bytes : 128;
    prm.nchunks = row_bytes / prm.kb;
    prm.rows = m == 256 ? 256 : 128;
    const int64_t total_rows = count * m;
    prm.jobs = (total_rows + prm.rows - 1) / prm.rows;
    prm.idesc_n128 = idesc(bf16, 128);
    prm.idesc_n256 = idesc(bf16, 256);
    prm.layout = prm.kb == 128 ? 2u : prm.kb == 64 ? 4u : 6u;  // 128B, 64B, 32B swizzle
    prm.fit = fit + first;
    prm.err = err;

    CUtensorMap map;
    const cuuint64_t dims[2] = {(cuuint64_t)m, (cuuint64_t)total_rows};
    const cuuint64_t strides[1] = {(cuuint64_t)row_bytes};
    const cuuint32_t box[2] = {(cuuint32_t)(prm.kb / esize), 128u};
    const cuuint32_t estr[2] = {1u, 1u};
    const CUtensorMapSwizzle sw = prm.kb == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                                  : prm.kb == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                                 : CU_TENSOR_MAP_SWIZZLE_32B;
    const uint8_t *base = (const uint8_t *)pop + (size_t)first * m * row_bytes;
    CUresult r = encode_fn()(&map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 2,
                             (void *)base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    if (!err) {
        // the launch's error word starts at zero
        void *addr = nullptr;
        cudaError_t e0 = cudaGetSymbolAddress(&addr, g_tc_err);
        if (e0 == cudaSuccess)
            e0 = cudaMemsetAsync(addr, 0, sizeof(uint32_t), s);
        if (e0 != cudaSuccess)
            return e0;
    }
    {
        const uint32_t sb = (uint32_t)prm.rows * (uint32_t)prm.kb;
        uint32_t ns = kRingBytes / sb;
        prm.nstages = (int32_t)(ns > (uint32_t)kMaxStages ? kMaxStages : ns);
    }
    const size_t smem = (size_t)prm.nstages * prm.rows * prm.kb + 1024;
    auto kern = bf16 ? (m == 256 ? k_fsq_tc<true, false> : k_fsq_tc<true, true>)
                     : (m == 256 ? k_fsq_tc<false, false> : k_fsq_tc<false, true>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t grid = prm.jobs < sms ? prm.jobs : sms;
    // m = 256 has a single issuer: no second MMA warp
    const int threads = m == 256 ? kTcThreads - 32 : kTcThreads;
    kern<<<(unsigned)grid, threads, smem, s>>>(map, prm);
    note_launches(1);
    return cudaGetLastError();
}

} // namespace hadga
