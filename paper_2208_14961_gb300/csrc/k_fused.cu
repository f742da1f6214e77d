// k_fused.cu -- the fused persistent generation kernel: every step of the
// population step (a2-a8; Sec. 3, the enumerated GA loop; Sec. 6, the loop of
// the listing) for one or more populations, generation after generation, in
// one cooperative launch.  Results are bit-identical to the one-kernel-per-
// operator path.
//
// Per generation g (all CTAs resident; two grid barriers):
//  Phase A  select.  The selection histogram of the population entering g
//           was filled by the previous generation's build phase (buckets
//           f >> shift for f <= cap, cap = previous threshold, which bounds
//           every survivor).  Each CTA scans it (one warp per population) to
//           find the threshold T of the 2N smallest; a bucket is exact when
//           its width 2^shift does not exceed 2^v, v = trailing zeros of the
//           OR of all fitness values (all F are multiples of 2^v), otherwise
//           extra refinement passes narrow it.  Warps then write, per tile of
//           32 slots, ballot masks of F < T and F == T.
//  Phase B  build.  Each CTA scans the tile masks into shared memory
//           (survivors in slot order), then builds pairs: parents k, k+N are
//           survivors number pi(k), pi(k+N) of the precomputed survivor order
//           of generation g; crossover, mutation and fitness of both
//           offspring run in registers (m <= 32: two threads per pair, one
//           per offspring) or in shared memory (32 < m <= 128: a warp per
//           pair); the new population goes to the other ping-pong buffer and
//           the histogram, OR word and best key of generation g + 1 are
//           accumulated with warp-aggregated atomics.
// Data written inside the launch is read with ld.global.cg (L2) so no SM
// can see a stale L1 line across generations.
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace hadga {

namespace {

constexpr uint32_t FULL = 0xFFFFFFFFu;

struct PopSel {
    uint32_t cap, shift;  // histogram of the current generation: f >> shift for f <= cap
    uint32_t v;           // every current F is a multiple of 2^v
    uint32_t lo, need;    // candidate bucket [lo, lo + 2^sr) and survivors still to take there
    uint32_t sr;          // width exponent of the candidate bucket
    uint32_t exact;
    uint32_t T, take;     // threshold and number of F == T survivors
    uint32_t lb, eb;      // joint (F < T, F == T) counts before the first tile of the population
    uint32_t capn, shiftn;  // histogram parameters of the next generation
    uint32_t boff;          // offset of this population's block histogram (~0: none)
    uint32_t gen0;          // generation of the population before this launch
    uint32_t bor;           // block OR of the new fitness values
    unsigned long long bbest;  // block minimum of the new best keys
};

__device__ __forceinline__ uint32_t ldcg32(const uint32_t *p) { return __ldcg(p); }
__device__ __forceinline__ unsigned long long ldcg64(const unsigned long long *p) { return __ldcg(p); }

// smallest s with (cap >> s) < kHistR
__device__ __forceinline__ uint32_t shift_for(uint32_t cap)
{
    const int bl = 32 - __clz(cap);
    return bl > 12 ? (uint32_t)(bl - 12) : 0u;
}

__device__ __forceinline__ uint32_t ctz_or(uint32_t orv) { return orv ? (uint32_t)(__ffs(orv) - 1) : 31u; }

__device__ __forceinline__ uint32_t *hist_of(const FusedPop &p, int parity) { return p.state + parity * kHistR; }
__device__ __forceinline__ uint32_t *ref_of(const FusedPop &p, int level) { return p.state + (2 + level) * kHistR; }
__device__ __forceinline__ uint32_t *stat_of(const FusedPop &p) { return p.state + 5 * kHistR; }

// Whole warp: bucket b in [0, nb) of h where the running count first reaches
// `need` (1 <= need <= total), and the count before it.
__device__ void warp_find_bucket(const uint32_t *h, uint32_t nb, uint32_t need, uint32_t *err, uint32_t &b_out,
                                 uint32_t &before_out)
{
    const int lane = threadIdx.x & 31;
    const uint32_t per = (nb + 31u) >> 5;
    const uint32_t lo = (uint32_t)lane * per, hi = min(lo + per, nb);
    uint32_t sum = 0;
    for (uint32_t b = lo; b < hi; ++b)
        sum += ldcg32(h + b);
    const uint32_t incl = warp_incl_scan(sum, lane), excl = incl - sum;
    const uint32_t bal = __ballot_sync(FULL, excl < need && need <= incl);
    uint32_t bres = 0, before = 0;
    if (bal == 0u) {
        if (lane == 0)
            atomicOr(err, ERR_INTERNAL);
        b_out = 0;
        before_out = 0;
        return;
    }
    const int owner = __ffs(bal) - 1;
    if (lane == owner) {
        uint32_t run = excl;
        bres = hi - 1;
        for (uint32_t b = lo; b < hi; ++b) {
            const uint32_t c = ldcg32(h + b);
            if (run + c >= need) {
                bres = b;
                break;
            }
            run += c;
        }
        before = run;
    }
    b_out = __shfl_sync(FULL, bres, owner);
    before_out = __shfl_sync(FULL, before, owner);
}

// Warp-aggregated histogram increment (all lanes call; ok selects the lanes
// that add one to bucket key).
__device__ __forceinline__ void warp_hist_add(uint32_t *h, bool ok, uint32_t key)
{
    const uint32_t k = ok ? key : 0xFFFFFFFFu;
    const uint32_t peers = __match_any_sync(FULL, k);
    const int lane = threadIdx.x & 31;
    if (ok && (__ffs(peers) - 1) == lane)
        atomicAdd(h + key, (uint32_t)__popc(peers));
}

__device__ __forceinline__ uint32_t warp_or(uint32_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v |= __shfl_xor_sync(FULL, v, o);
    return v;
}

__device__ __forceinline__ uint32_t warp_max(uint32_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = max(v, __shfl_xor_sync(FULL, v, o));
    return v;
}

// Exclusive prefix sums over e in [0, n) of cnt(e) into out[e] (shared
// memory), each thread walking one contiguous chunk: two short sequential
// passes around a single block-wide scan.  Every thread calls.
template <class Cnt>
__device__ __forceinline__ void block_scan_chunks(uint32_t n, Cnt cnt, uint32_t *out, uint32_t *tmp)
{
    const uint32_t per = (n + blockDim.x - 1) / blockDim.x;
    const uint32_t lo = min(n, threadIdx.x * per), hi = min(n, lo + per);
    uint32_t sum = 0;
    for (uint32_t e = lo; e < hi; ++e)
        sum += cnt(e);
    uint32_t tot;
    uint32_t ex = block_excl_scan(sum, tmp, &tot);
    for (uint32_t e = lo; e < hi; ++e) {
        const uint32_t c = cnt(e);
        out[e] = ex;
        ex += c;
    }
    __syncthreads();
}

// Survivor bookkeeping of phase B, per tile t of the joint tile space:
//   tm[t] = (F < T mask) | (F == T mask) << 32
//   ex[t] = exclusive prefix over tiles of (popc(lt) << 32 | popc(eq))
// Within population i (bases lb, eb at its first tile) the survivors before
// tile t number (lt_before) + min(eq_before, take), and the tile's survivor
// mask is lt | the lowest (take - eq_before) bits of eq.
struct Surv {
    const unsigned long long *tm, *ex;
};

__device__ __forceinline__ uint32_t surv_before(const Surv &sv, uint32_t tt, const PopSel &S)
{
    const unsigned long long e = sv.ex[tt];
    const uint32_t ltb = (uint32_t)(e >> 32) - S.lb, eqb = (uint32_t)e - S.eb;
    return ltb + min(eqb, S.take);
}

// Slot of survivor number d of a population: binary search over the tile
// prefix, then a select-bit inside the tile.
__device__ __forceinline__ uint32_t survivor_of(uint32_t d, const FusedPop &p, const PopSel &S, const Surv &sv,
                                                uint32_t *err)
{
    const uint32_t tb = p.tile_base;
    uint32_t lo = 0, hi = p.ntiles - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (surv_before(sv, tb + mid, S) <= d)
            lo = mid;
        else
            hi = mid - 1;
    }
    const unsigned long long m64 = sv.tm[tb + lo];
    const uint32_t eqb = min((uint32_t)sv.ex[tb + lo] - S.eb, S.take);
    const uint32_t mask = (uint32_t)m64 | lowest_set_bits((uint32_t)(m64 >> 32), (int)(S.take - eqb));
    const uint32_t r = d - surv_before(sv, tb + lo, S);
    const uint32_t P = (uint32_t)(4 * p.N);
    if (r >= (uint32_t)__popc(mask)) {
        atomicOr(err, ERR_INTERNAL);
        return P - 1;
    }
    const uint32_t slot = lo * 32u + (uint32_t)nth_set_bit(mask, (int)r);
    return slot < P ? slot : P - 1;
}

// Slot of non-survivor number o (in slot order): tiles hold 32t slots before
// tile t, of which surv_before(t) survive.
__device__ __forceinline__ uint32_t nonsurvivor_of(uint32_t o, const FusedPop &p, const PopSel &S, const Surv &sv,
                                                   uint32_t *err)
{
    const uint32_t tb = p.tile_base;
    uint32_t lo = 0, hi = p.ntiles - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (32u * mid - surv_before(sv, tb + mid, S) <= o)
            lo = mid;
        else
            hi = mid - 1;
    }
    const unsigned long long m64 = sv.tm[tb + lo];
    const uint32_t eqb = min((uint32_t)sv.ex[tb + lo] - S.eb, S.take);
    const uint32_t surv = (uint32_t)m64 | lowest_set_bits((uint32_t)(m64 >> 32), (int)(S.take - eqb));
    const uint32_t P = (uint32_t)(4 * p.N);
    const uint32_t tail = P - 32u * lo;
    const uint32_t valid = tail >= 32u ? 0xFFFFFFFFu : ((1u << tail) - 1u);
    const uint32_t mask = valid & ~surv;
    const uint32_t r = o - (32u * lo - surv_before(sv, tb + lo, S));
    if (r >= (uint32_t)__popc(mask)) {
        atomicOr(err, ERR_INTERNAL);
        return P - 1;
    }
    return 32u * lo + (uint32_t)nth_set_bit(mask, (int)r);
}

// Draws of one build item that do not depend on the selection: survivor
// number d, cut point c and (for NC = NR = 1) the mutated column and rows.
struct Pre {
    uint32_t d, c, cc, ra, rb;
};

__device__ __forceinline__ Pre make_pre(const FusedPop &p, uint32_t gen, uint32_t tch, uint32_t k, int half)
{
    const uint32_t N = (uint32_t)p.N;
    Pre r;
    r.d = __ldg(p.perm + (size_t)tch * 2u * N + k + (half ? N : 0u));
    r.c = (uint32_t)cut_point(p.seed, p.pop_id, gen, k, p.m);
    r.cc = r.ra = r.rb = 0u;
    if (p.NC == 1 && p.NR == 1) {
        const uint4 w = philox_block(p.seed, p.pop_id, OP_MUTATE, gen, k + (half ? N : 0u), 0u, 0u);
        r.cc = uniform_int(w.x, 1u, (uint32_t)(p.m - 1));
        r.ra = uniform_int(w.y, 0u, (uint32_t)(p.m - 1));
        r.rb = uniform_int(w.z, 0u, (uint32_t)(p.m - 1));
    }
    return r;
}

// Mutation draws of offspring o: NC columns, NR first rows, NR second rows.
struct Draws {
    uint32_t seed, pop_id, gen, o, block;
    uint4 cur;
    int used;
    __device__ Draws(uint32_t s, uint32_t p, uint32_t g, uint32_t oo)
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

template <int M, int KIND>
__device__ __forceinline__ uint32_t fitness_regs(const uint32_t (&c)[M])
{
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < M; ++i) {
#pragma unroll
        for (int j = i + 1; j < M; ++j)
            acc += fit_term<KIND>(M - 2 * __popc(c[i] ^ c[j]));
    }
    return fit_finish<KIND>(acc);
}

// ---------------------------------------------------------------------------
// m <= 32: two threads per pair (lane pair 2j, 2j+1), thread `half` builds
// offspring O_{1 + half}; its parent is P_1 (half 0) or P_2 (half 1).
// ---------------------------------------------------------------------------
template <int M>
__device__ __forceinline__ void pair_thread(const FusedPop &p, const PopSel &S, int src, uint32_t gen, const Pre &pre,
                                            uint32_t k, int half, bool valid, const Surv &sv, uint32_t *err,
                                            uint32_t &f_par, uint32_t &slot_par, uint32_t &f_child,
                                            uint32_t &slot_child)
{
    const uint32_t N = (uint32_t)p.N;
    uint32_t s_mine = 0;
    if (valid)
        s_mine = survivor_of(pre.d, p, S, sv, err);
    const uint32_t s_other = __shfl_xor_sync(FULL, s_mine, 1);
    if (!valid)
        return;
    const uint32_t s1 = half ? s_other : s_mine, s2 = half ? s_mine : s_other;
    const uint32_t *src_pop = p.pop[src];
    uint32_t *dst_pop = p.pop[src ^ 1];
    uint32_t p1[M], p2[M];
    const uint4 *a = reinterpret_cast<const uint4 *>(src_pop + (size_t)s1 * M);
    const uint4 *b = reinterpret_cast<const uint4 *>(src_pop + (size_t)s2 * M);
#pragma unroll
    for (int v = 0; v < M / 4; ++v) {
        const uint4 x = __ldcg(a + v), y = __ldcg(b + v);
        p1[4 * v] = x.x, p1[4 * v + 1] = x.y, p1[4 * v + 2] = x.z, p1[4 * v + 3] = x.w;
        p2[4 * v] = y.x, p2[4 * v + 1] = y.y, p2[4 * v + 2] = y.z, p2[4 * v + 3] = y.w;
    }
    f_par = ldcg32(p.fit[src] + s_mine);
    slot_par = half ? k + N : k;
    {
        uint4 *d = reinterpret_cast<uint4 *>(dst_pop + (size_t)slot_par * M);
#pragma unroll
        for (int v = 0; v < M / 4; ++v) {
            const uint32_t *q = half ? p2 : p1;
            d[v] = make_uint4(q[4 * v], q[4 * v + 1], q[4 * v + 2], q[4 * v + 3]);
        }
        p.fit[src ^ 1][slot_par] = f_par;
    }
    // crossover (Sec. 3.4): O1 = P1[:, :c] | P2[:, c:], O2 = P2[:, :c] | P1[:, c:]
    const int c = (int)pre.c;
    uint32_t o[M];
#pragma unroll
    for (int j = 0; j < M; ++j)
        o[j] = ((j < c) != (half != 0)) ? p1[j] : p2[j];
    // mutation (Sec. 3.5): columns in order, pairs in order, flip iff different
    {
        Draws dr(p.seed, p.pop_id, gen, k + (half ? N : 0u));
        const int NC = p.NC, NR = p.NR;
        if (NC == 1 && NR == 1) {
            const uint32_t cc = pre.cc, ra = pre.ra, rb = pre.rb;
#pragma unroll
            for (int j = 1; j < M; ++j) {
                if ((uint32_t)j == cc) {
                    const uint32_t t = ((o[j] >> ra) ^ (o[j] >> rb)) & 1u;
                    o[j] ^= (t << ra) | (t << rb);
                }
            }
        } else {
            uint8_t cols[64], r1[64], r2[64];
            for (int jc = 0; jc < NC; ++jc)
                cols[jc] = (uint8_t)uniform_int(dr.next(), 1u, (uint32_t)(M - 1));
            for (int ir = 0; ir < NR; ++ir)
                r1[ir] = (uint8_t)uniform_int(dr.next(), 0u, (uint32_t)(M - 1));
            for (int ir = 0; ir < NR; ++ir)
                r2[ir] = (uint8_t)uniform_int(dr.next(), 0u, (uint32_t)(M - 1));
            for (int jc = 0; jc < NC; ++jc) {
                const int cc = cols[jc];
                uint32_t w = 0;
#pragma unroll
                for (int j = 1; j < M; ++j)
                    w = (j == cc) ? o[j] : w;
                for (int ir = 0; ir < NR; ++ir) {
                    const uint32_t ra = r1[ir], rb = r2[ir];
                    const uint32_t t = ((w >> ra) ^ (w >> rb)) & 1u;
                    w ^= (t << ra) | (t << rb);
                }
#pragma unroll
                for (int j = 1; j < M; ++j)
                    o[j] = (j == cc) ? w : o[j];
            }
        }
    }
    uint32_t f;
    switch (p.kind) {
    case FIT_SQ: f = fitness_regs<M, FIT_SQ>(o); break;
    case FIT_ABS: f = fitness_regs<M, FIT_ABS>(o); break;
    default: f = fitness_regs<M, FIT_NNZ>(o); break;
    }
    slot_child = 2u * N + k + (half ? N : 0u);
    {
        uint4 *d = reinterpret_cast<uint4 *>(dst_pop + (size_t)slot_child * M);
#pragma unroll
        for (int v = 0; v < M / 4; ++v)
            d[v] = make_uint4(o[4 * v], o[4 * v + 1], o[4 * v + 2], o[4 * v + 3]);
        p.fit[src ^ 1][slot_child] = f;
    }
    f_child = f;
}

// ---------------------------------------------------------------------------
// a7 -- incremental fitness of one offspring (warp-wide; not in the paper,
// which recomputes G: derived from the fitness of Sec. 3.2 under the
// operators of Sec. 3.4 and 3.5).  Its Gram / 2, h,
// is assembled in its own buffer from the parents' buffers: entries with
// j < c from the parent giving the first c columns (gt), entries with i >= c
// from the other (gbm), the c(m - c) cross entries recomputed from the column
// bits (ct: first-part columns, cb: second-part columns).  Then the mutation
// runs flip by flip: a successful flip of rows r1, r2 in column cc changes
// only row/column cc of G (by -2s(Q[r1][j] - Q[r2][j]), s = Q[r1][cc]), so
// those m - 1 entries and the fitness are updated and the two bits flipped
// in the offspring's columns `bo` (which hold the crossover result on entry).
// The fitness is the sum of the per-entry terms, kept up to date on the way.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int tri_index(int i, int j, int m) { return i * (m - 1) - (i * (i - 1)) / 2 + (j - i - 1); }

__device__ __forceinline__ uint32_t mutation_word(const FusedPop &p, uint32_t gen, uint32_t o, int w)
{
    return word_of(philox_block(p.seed, p.pop_id, OP_MUTATE, gen, o, 0u, (uint32_t)(w >> 2)), w & 3);
}

template <int W, int KIND>
__device__ uint32_t offspring_incremental(const FusedPop &p, uint32_t *bo, const uint32_t *ct, const uint32_t *cb,
                                          int c, uint32_t gt, uint32_t gbm, uint32_t go, uint32_t gen, uint32_t o,
                                          int lane)
{
    const int m = p.m, half_m = m >> 1;
    const int8_t *Gt = p.gram + (size_t)gt * p.dpad;
    const int8_t *Gb = p.gram + (size_t)gbm * p.dpad;
    int8_t *Go = p.gram + (size_t)go * p.dpad;
    uint32_t acc = 0;
    int base = 0;
    for (int i = 0; i < m - 1; ++i) {
        const int L = m - 1 - i;
        for (int jj = lane; jj < L; jj += 32) {
            const int j = i + 1 + jj;
            int h;
            if (j < c) {
                h = (int)__ldcg(reinterpret_cast<const signed char *>(Gt + base + jj));
            } else if (i >= c) {
                h = (int)__ldcg(reinterpret_cast<const signed char *>(Gb + base + jj));
            } else {
                int d = 0;
#pragma unroll
                for (int w = 0; w < W; ++w)
                    d += __popc(ct[i * W + w] ^ cb[j * W + w]);
                h = half_m - d;
            }
            __stcg(reinterpret_cast<signed char *>(Go) + base + jj, (signed char)h);
            acc += fit_term<KIND>(2 * h);
        }
        base += L;
    }
    __syncwarp();
    // mutation, flip by flip; draw word w of offspring o (NC columns, then NR
    // first rows, then NR second rows) is word w mod 4 of block w / 4
    const int NC = p.NC, NR = p.NR;
    for (int jc = 0; jc < NC; ++jc) {
        const int cc = (int)uniform_int(mutation_word(p, gen, o, jc), 1u, (uint32_t)(m - 1));
        uint32_t *col = bo + cc * W;
        for (int ir = 0; ir < NR; ++ir) {
            const int ra = (int)uniform_int(mutation_word(p, gen, o, NC + ir), 0u, (uint32_t)(m - 1));
            const int rb = (int)uniform_int(mutation_word(p, gen, o, NC + NR + ir), 0u, (uint32_t)(m - 1));
            const int ba = (int)((col[ra >> 5] >> (ra & 31)) & 1u), bb = (int)((col[rb >> 5] >> (rb & 31)) & 1u);
            if (ba == bb)
                continue;  // equal entries: no flip (the same on every lane)
            const int s = ba ? -1 : 1;  // Q[r1][cc] before the flip
            for (int j = lane; j < m; j += 32) {
                if (j == cc)
                    continue;
                const int qa = ((bo[j * W + (ra >> 5)] >> (ra & 31)) & 1u) ? -1 : 1;
                const int qb = ((bo[j * W + (rb >> 5)] >> (rb & 31)) & 1u) ? -1 : 1;
                if (qa == qb)
                    continue;
                signed char *e = reinterpret_cast<signed char *>(Go) + (cc < j ? tri_index(cc, j, m) : tri_index(j, cc, m));
                const int h0 = (int)__ldcg(e);
                const int h1 = h0 - s * (qa - qb);  // G moves by -2s(qa - qb)
                __stcg(e, (signed char)h1);
                acc += fit_term<KIND>(2 * h1) - fit_term<KIND>(2 * h0);
            }
            __syncwarp();
            if (lane == 0) {
                col[ra >> 5] ^= 1u << (ra & 31);
                col[rb >> 5] ^= 1u << (rb & 31);
            }
            __syncwarp();
        }
    }
    return fit_finish<KIND>(warp_sum(acc));
}

// ---------------------------------------------------------------------------
// 32 < m <= 128: a warp per pair, matrices staged in shared memory.
// ---------------------------------------------------------------------------
template <int W>
__device__ void pair_warp(const FusedPop &p, PopSel &S, int src, uint32_t gen, uint32_t tch, uint32_t k,
                          const Surv &sv, uint32_t *err, uint32_t *buf, uint32_t *hist_next, uint32_t *bhist)
{
    const int lane = threadIdx.x & 31;
    const int m = p.m;
    const uint32_t N = (uint32_t)p.N, words = (uint32_t)(m * W);
    uint32_t s1 = 0, s2 = 0, F1 = 0, F2 = 0;
    int c = 1;
    if (lane == 0) {
        const uint32_t *row = p.perm + (size_t)tch * 2u * N;
        s1 = survivor_of(__ldg(row + k), p, S, sv, err);
        s2 = survivor_of(__ldg(row + k + N), p, S, sv, err);
        F1 = ldcg32(p.fit[src] + s1);
        F2 = ldcg32(p.fit[src] + s2);
        c = cut_point(p.seed, p.pop_id, gen, k, m);
    }
    s1 = __shfl_sync(FULL, s1, 0);
    s2 = __shfl_sync(FULL, s2, 0);
    c = __shfl_sync(FULL, c, 0);
    // incremental mode: parents keep their Gram buffers, offspring take the
    // buffers of the non-survivors k and k + N (in slot order)
    const bool inc = p.gram != nullptr;
    uint32_t gb1 = 0, gb2 = 0, go0 = 0, go1 = 0;
    if (inc && lane == 0) {
        gb1 = ldcg32(p.gidx[src] + s1);
        gb2 = ldcg32(p.gidx[src] + s2);
        go0 = ldcg32(p.gidx[src] + nonsurvivor_of(k, p, S, sv, err));
        go1 = ldcg32(p.gidx[src] + nonsurvivor_of(k + N, p, S, sv, err));
        const uint32_t P = (uint32_t)(4 * p.N);
        if ((gb1 | gb2 | go0 | go1) >= P && (gb1 >= P || gb2 >= P || go0 >= P || go1 >= P)) {
            atomicOr(err, ERR_INTERNAL);  // never expected: indices stay a permutation of [0, P)
            gb1 = gb1 < P ? gb1 : 0u;
            gb2 = gb2 < P ? gb2 : 0u;
            go0 = go0 < P ? go0 : 0u;
            go1 = go1 < P ? go1 : 0u;
        }
        p.gidx[src ^ 1][k] = gb1;
        p.gidx[src ^ 1][k + N] = gb2;
        p.gidx[src ^ 1][2u * N + k] = go0;
        p.gidx[src ^ 1][3u * N + k] = go1;
    }
    if (inc) {
        gb1 = __shfl_sync(FULL, gb1, 0);
        gb2 = __shfl_sync(FULL, gb2, 0);
        go0 = __shfl_sync(FULL, go0, 0);
        go1 = __shfl_sync(FULL, go1, 0);
    }
    uint32_t *b1 = buf, *b2 = buf + words, *bo = buf + 2 * words;
    const uint32_t *sp = p.pop[src];
    uint32_t *dp = p.pop[src ^ 1];
    for (uint32_t e = lane; e < words; e += 32) {
        const uint32_t x = ldcg32(sp + (size_t)s1 * words + e), y = ldcg32(sp + (size_t)s2 * words + e);
        b1[e] = x;
        b2[e] = y;
        dp[(size_t)k * words + e] = x;
        dp[(size_t)(k + N) * words + e] = y;
    }
    if (lane == 0) {
        p.fit[src ^ 1][k] = F1;
        p.fit[src ^ 1][k + N] = F2;
    }
    uint32_t fc[2] = {0, 0};
    for (int half = 0; half < 2; ++half) {
        __syncwarp();
        for (uint32_t e = lane; e < words; e += 32)
            bo[e] = (((int)(e / W) < c) != (half != 0)) ? b1[e] : b2[e];
        __syncwarp();
        if (inc) {
            uint32_t f;
            switch (p.kind) {
            case FIT_SQ: f = offspring_incremental<W, FIT_SQ>(p, bo, half ? b2 : b1, half ? b1 : b2, c, half ? gb2 : gb1, half ? gb1 : gb2, half ? go1 : go0, gen, k + (half ? N : 0u), lane); break;
            case FIT_ABS: f = offspring_incremental<W, FIT_ABS>(p, bo, half ? b2 : b1, half ? b1 : b2, c, half ? gb2 : gb1, half ? gb1 : gb2, half ? go1 : go0, gen, k + (half ? N : 0u), lane); break;
            default: f = offspring_incremental<W, FIT_NNZ>(p, bo, half ? b2 : b1, half ? b1 : b2, c, half ? gb2 : gb1, half ? gb1 : gb2, half ? go1 : go0, gen, k + (half ? N : 0u), lane); break;
            }
            const uint32_t slot = 2u * N + k + (half ? N : 0u);
            for (uint32_t e = lane; e < words; e += 32)
                dp[(size_t)slot * words + e] = bo[e];
            if (lane == 0)
                p.fit[src ^ 1][slot] = f;
            fc[half] = f;
            continue;
        }
        if (lane == 0) {
            Draws dr(p.seed, p.pop_id, gen, k + (half ? N : 0u));
            uint8_t cols[64], r1[64], r2[64];
            for (int jc = 0; jc < p.NC; ++jc)
                cols[jc] = (uint8_t)uniform_int(dr.next(), 1u, (uint32_t)(m - 1));
            for (int ir = 0; ir < p.NR; ++ir)
                r1[ir] = (uint8_t)uniform_int(dr.next(), 0u, (uint32_t)(m - 1));
            for (int ir = 0; ir < p.NR; ++ir)
                r2[ir] = (uint8_t)uniform_int(dr.next(), 0u, (uint32_t)(m - 1));
            for (int jc = 0; jc < p.NC; ++jc) {
                uint32_t *col = bo + cols[jc] * W;
                for (int ir = 0; ir < p.NR; ++ir) {
                    const int ra = r1[ir], rb = r2[ir];
                    const uint32_t ba = (col[ra >> 5] >> (ra & 31)) & 1u, bb = (col[rb >> 5] >> (rb & 31)) & 1u;
                    if (ba != bb) {
                        col[ra >> 5] ^= 1u << (ra & 31);
                        col[rb >> 5] ^= 1u << (rb & 31);
                    }
                }
            }
        }
        __syncwarp();
        uint32_t f;
        switch (p.kind) {
        case FIT_SQ: f = warp_fitness_cols<W, FIT_SQ>(bo, m, lane); break;
        case FIT_ABS: f = warp_fitness_cols<W, FIT_ABS>(bo, m, lane); break;
        default: f = warp_fitness_cols<W, FIT_NNZ>(bo, m, lane); break;
        }
        const uint32_t slot = 2u * N + k + (half ? N : 0u);
        for (uint32_t e = lane; e < words; e += 32)
            dp[(size_t)slot * words + e] = bo[e];
        if (lane == 0)
            p.fit[src ^ 1][slot] = f;
        fc[half] = f;
    }
    if (lane == 0) {
        const uint32_t fv[4] = {F1, F2, fc[0], fc[1]};
        const uint32_t slots[4] = {k, k + N, 2u * N + k, 3u * N + k};
        unsigned long long bk = ~0ull;
        uint32_t orr = 0;
        for (int i = 0; i < 4; ++i) {
            if (fv[i] <= S.capn)
                atomicAdd((S.boff != 0xFFFFFFFFu ? bhist + S.boff : hist_next) + (fv[i] >> S.shiftn), 1u);
            orr |= fv[i];
            const unsigned long long key = ((unsigned long long)fv[i] << 32) | slots[i];
            bk = key < bk ? key : bk;
        }
        atomicOr(&S.bor, orr);
        atomicMin(&S.bbest, bk);
    }
    __syncwarp();
}

__device__ __forceinline__ unsigned long long warp_incl_scan_u64(unsigned long long v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(FULL, v, o);
        if (lane >= o)
            v += t;
    }
    return v;
}

// Exclusive prefix of cnt(e) over e in [0, n) into out[e] (shared memory),
// 64-bit, one contiguous chunk per thread, one block-wide scan.
template <class Cnt>
__device__ __forceinline__ void block_scan_chunks_u64(uint32_t n, Cnt cnt, unsigned long long *out,
                                                      unsigned long long *tmp)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    const uint32_t per = (n + blockDim.x - 1) / blockDim.x;
    const uint32_t lo = min(n, threadIdx.x * per), hi = min(n, lo + per);
    unsigned long long sum = 0;
    for (uint32_t e = lo; e < hi; ++e)
        sum += cnt(e);
    const unsigned long long inc = warp_incl_scan_u64(sum, lane);
    if (lane == 31)
        tmp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const unsigned long long w = lane < nw ? tmp[lane] : 0ull;
        const unsigned long long wi = warp_incl_scan_u64(w, lane);
        if (lane < nw)
            tmp[lane] = wi - w;
    }
    __syncthreads();
    unsigned long long ex = tmp[warp] + inc - sum;
    for (uint32_t e = lo; e < hi; ++e) {
        const unsigned long long c = cnt(e);
        out[e] = ex;
        ex += c;
    }
    __syncthreads();
}

// Population owning joint index x given increasing bases (linear: npop <= 16).
template <class Base>
__device__ __forceinline__ int owner_of(uint32_t x, int npop, Base base)
{
    int i = 0;
    while (i + 1 < npop && x >= base(i + 1))
        ++i;
    return i;
}

} // namespace

__global__ void __launch_bounds__(kFusedThreads, 1) k_fused(const __grid_constant__ FusedParams prm)
{
    extern __shared__ __align__(16) uint32_t dyn[];
    __shared__ PopSel S[kMaxPops];
    __shared__ uint32_t s_tmp[33];
    __shared__ unsigned long long s_tmp64[32];
    __shared__ uint32_t hoff[kMaxPops];
    __shared__ int s_flag;

    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    const int npop = prm.npop;
    const uint32_t nblocks = gridDim.x;
    const uint32_t gtid = blockIdx.x * blockDim.x + tid, gthreads = nblocks * blockDim.x;
    // warps enumerated across blocks first, so consecutive work items land on
    // different SMs
    const uint32_t gwarp = (uint32_t)wib * nblocks + blockIdx.x, gwarps = gthreads >> 5;
    const uint32_t TT = prm.total_tiles;
    // shared layout: [tile masks and their prefix (phase B) | staged
    // histograms (phase A)] [warp buffers]
    const uint32_t r1 = max(4u * TT, 2u * kHistSmem);
    unsigned long long *tm = reinterpret_cast<unsigned long long *>(dyn);
    unsigned long long *ex = tm + TT;
    uint32_t *hcnt = dyn, *hpre = dyn + kHistSmem;
    uint32_t *bhist = dyn + r1;  // block-local histograms of the next generation
    uint32_t *wbuf = bhist + kHistSmem + wib * prm.warp_buf_words;
    const Surv sv{tm, ex};
    uint32_t *err = prm.err;
    uint32_t epoch = 0;
    int src = prm.src;
    int done = 0;
    auto tile_base = [&](int i) { return prm.p[i].tile_base; };

    // ---- pre-pass: max and OR of the current fitness of every population -----
    {
        const int par0 = 0;  // buffers alternate with the generation index inside the launch
        if (tid < npop)
            S[tid].gen0 = ldcg32(prm.p[tid].gen_dev);
        for (int i = 0; i < npop; ++i) {
            const FusedPop &p = prm.p[i];
            const uint32_t P = (uint32_t)(4 * p.N);
            uint32_t mx = 0, orr = 0;
            for (uint32_t q = gtid; q < P; q += gthreads) {
                const uint32_t f = ldcg32(p.fit[src] + q);
                mx = max(mx, f);
                orr |= f;
            }
            mx = warp_max(mx);
            orr = warp_or(orr);
            if (lane == 0) {
                atomicMax(stat_of(p) + 0, mx);
                atomicOr(stat_of(p) + 1 + par0, orr);
            }
        }
        if (!grid_barrier(prm.bar, nblocks, epoch, err))
            return;
        if (tid < npop) {
            const FusedPop &p = prm.p[tid];
            const uint32_t cap = ldcg32(stat_of(p) + 0);
            const uint32_t v = ctz_or(ldcg32(stat_of(p) + 1 + par0));
            S[tid].cap = cap;
            S[tid].shift = max(v, shift_for(cap));
        }
        __syncthreads();
        for (int i = 0; i < npop; ++i) {
            const FusedPop &p = prm.p[i];
            const uint32_t P = (uint32_t)(4 * p.N);
            uint32_t *h = hist_of(p, par0);
            const uint32_t cap = S[i].cap, sh = S[i].shift;
            // uniform trip count so the warp-collective add stays converged
            const uint32_t span = (P + 31u) & ~31u;
            for (uint32_t q = gtid; q < ((span + gthreads - 1) / gthreads) * gthreads; q += gthreads) {
                const bool in = q < P;
                const uint32_t f = in ? ldcg32(p.fit[src] + q) : 0u;
                warp_hist_add(h, in && f <= cap, f >> sh);
            }
        }
        if (!grid_barrier(prm.bar, nblocks, epoch, err))
            return;
    }

    uint32_t ref_level = 0;
    for (int t = 0; t < prm.ngen; ++t) {
        const int par = t & 1;

        // ---- phase A: threshold of the 2N smallest ---------------------------------
        // first tile of this warp: its fitness is loaded now, with the histograms
        uint32_t f_pre = 0;
        int i_pre = 0;
        if (gwarp < TT) {
            i_pre = owner_of(gwarp, npop, tile_base);
            const FusedPop &p = prm.p[i_pre];
            const uint32_t q = (gwarp - p.tile_base) * 32u + lane;
            f_pre = q < (uint32_t)(4 * p.N) ? ldcg32(p.fit[src] + q) : 0u;
        }
        if (tid < npop) {
            PopSel &s = S[tid];
            s.v = ctz_or(ldcg32(stat_of(prm.p[tid]) + 1 + par));
            s.need = 0xFFFFFFFFu;  // marks "crossing not found"
        }
        for (int i = 0; i < npop; ++i) {
            uint32_t *hn = hist_of(prm.p[i], par ^ 1);
            for (uint32_t e = gtid; e < (uint32_t)kHistR; e += gthreads)
                hn[e] = 0u;
        }
        if (blockIdx.x == 0 && tid < npop) {
            const FusedPop &p = prm.p[tid];
            stat_of(p)[1 + (par ^ 1)] = 0u;
            p.traj[(S[tid].gen0 + (uint32_t)t) % (uint32_t)p.traj_cap] = ~0ull;
        }
        // histograms staged in shared memory (groups of populations that fit),
        // scanned in one block-wide pass, crossing of 2N located per population
        for (int i0 = 0; i0 < npop;) {
            uint32_t off = 0;
            int i1 = i0;
            while (i1 < npop) {
                const uint32_t nb = (S[i1].cap >> S[i1].shift) + 1u;
                if (i1 > i0 && off + nb > kHistSmem)
                    break;
                if (tid == 0)
                    hoff[i1] = off;
                off += nb;
                ++i1;
            }
            __syncthreads();
            for (uint32_t e = tid; e < off; e += blockDim.x) {
                int i = i0;
                while (i + 1 < i1 && e >= hoff[i + 1])
                    ++i;
                hcnt[e] = ldcg32(hist_of(prm.p[i], par) + (e - hoff[i]));
            }
            __syncthreads();
            block_scan_chunks(off, [&](uint32_t e) { return hcnt[e]; }, hpre, s_tmp);
            for (uint32_t e = tid; e < off; e += blockDim.x) {
                int i = i0;
                while (i + 1 < i1 && e >= hoff[i + 1])
                    ++i;
                const uint32_t need = (uint32_t)(2 * prm.p[i].N);
                const uint32_t x = hpre[e] - hpre[hoff[i]], h = hcnt[e];
                if (h && x < need && need <= x + h) {
                    S[i].lo = (e - hoff[i]) << S[i].shift;
                    S[i].need = need - x;
                }
            }
            __syncthreads();
            i0 = i1;
        }
        if (tid == 0)
            s_flag = 0;
        if (tid < npop) {
            PopSel &s = S[tid];
            if (s.need == 0xFFFFFFFFu) {
                atomicOr(err, ERR_INTERNAL);
                s.lo = 0;
                s.need = 1;
            }
            s.sr = s.shift;
            s.exact = s.shift <= s.v ? 1u : 0u;
        }
        __syncthreads();
        if (tid < npop && !S[tid].exact)
            atomicOr(&s_flag, 1);
        __syncthreads();
        // refinement passes while a candidate bucket may hold several values
        while (s_flag) {
            const int rl = (int)(ref_level % 3u), rz = (int)((ref_level + 1u) % 3u);
            for (int i = 0; i < npop; ++i) {
                const FusedPop &p = prm.p[i];
                uint32_t *hz = ref_of(p, rz);
                for (uint32_t e = gtid; e < (uint32_t)kHistR; e += gthreads)
                    hz[e] = 0u;
                if (S[i].exact)
                    continue;
                const uint32_t P = (uint32_t)(4 * p.N);
                const uint32_t lo = S[i].lo, sr = S[i].sr;
                const uint32_t sn = max(S[i].v, sr > 12u ? sr - 12u : 0u);
                uint32_t *h = ref_of(p, rl);
                const uint32_t span = (P + 31u) & ~31u;
                for (uint32_t q = gtid; q < ((span + gthreads - 1) / gthreads) * gthreads; q += gthreads) {
                    const bool in = q < P;
                    const uint32_t f = in ? ldcg32(p.fit[src] + q) : 0u;
                    const bool hit = in && f >= lo && ((uint64_t)(f - lo) >> sr) == 0u;
                    warp_hist_add(h, hit, hit ? (f - lo) >> sn : 0u);
                }
            }
            if (!grid_barrier(prm.bar, nblocks, epoch, err))
                return;
            if (wib < npop && !S[wib].exact) {
                const FusedPop &p = prm.p[wib];
                PopSel &s = S[wib];
                const uint32_t sn = max(s.v, s.sr > 12u ? s.sr - 12u : 0u);
                uint32_t b, before;
                warp_find_bucket(ref_of(p, rl), 1u << (s.sr - sn), s.need, err, b, before);
                if (lane == 0) {
                    s.lo += b << sn;
                    s.need -= before;
                    s.sr = sn;
                    s.exact = sn <= s.v ? 1u : 0u;
                }
            }
            ++ref_level;
            __syncthreads();
            if (tid == 0) {
                int any = 0;
                for (int i = 0; i < npop; ++i)
                    any |= S[i].exact ? 0 : 1;
                s_flag = any;
            }
            __syncthreads();
        }
        if (tid < npop) {
            PopSel &s = S[tid];
            s.T = s.lo;
            s.take = s.need;
            s.capn = s.T;
            s.shiftn = max(s.v, shift_for(s.T));
            s.bor = 0u;
            s.bbest = ~0ull;
        }
        __syncthreads();
        if (tid == 0) {
            uint32_t off = 0;
            for (int i = 0; i < npop; ++i) {
                const uint32_t nb = (S[i].capn >> S[i].shiftn) + 1u;
                S[i].boff = off + nb <= kHistSmem ? off : 0xFFFFFFFFu;
                if (off + nb <= kHistSmem)
                    off += nb;
            }
        }
        // selection-independent draws of this warp's first build item, computed
        // while the other blocks catch up
        Pre pre0{0u, 1u, 1u, 0u, 0u};
        const uint32_t nwork_t = prm.thread_slots >> 5;
        if (gwarp < nwork_t) {
            const uint32_t u = gwarp * 32u + (uint32_t)lane;
            int i = -1;
            for (int j = 0; j < npop; ++j)
                if (prm.p[j].m <= 32 && u >= prm.p[j].work_base)
                    i = (i < 0 || prm.p[j].work_base >= prm.p[i].work_base) ? j : i;
            if (i >= 0) {
                const FusedPop &p = prm.p[i];
                const uint32_t local = u - p.work_base, k = local >> 1;
                if (k < (uint32_t)p.N)
                    pre0 = make_pre(p, S[i].gen0 + 1u + (uint32_t)t, (uint32_t)t, k, (int)(local & 1u));
            }
        }
        // tile masks: F < T and F == T per 32 slots
        for (uint32_t tl = gwarp; tl < TT; tl += gwarps) {
            const int i = tl == gwarp ? i_pre : owner_of(tl, npop, tile_base);
            const FusedPop &p = prm.p[i];
            const uint32_t P = (uint32_t)(4 * p.N), T = S[i].T;
            const uint32_t q = (tl - p.tile_base) * 32u + lane;
            const uint32_t f = tl == gwarp ? f_pre : (q < P ? ldcg32(p.fit[src] + q) : 0u);
            const uint32_t lt = __ballot_sync(FULL, q < P && f < T);
            const uint32_t eq = __ballot_sync(FULL, q < P && f == T);
            if (lane == 0)
                p.tmask[tl - p.tile_base] = (unsigned long long)lt | ((unsigned long long)eq << 32);
        }
        if (!grid_barrier(prm.bar, nblocks, epoch, err))
            return;

        // ---- phase B: survivors in slot order, then build ------------------------
        for (uint32_t t0 = tid; t0 < TT; t0 += 4u * blockDim.x) {
            unsigned long long v[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const uint32_t tt = t0 + (uint32_t)r * blockDim.x;
                if (tt < TT) {
                    const int i = owner_of(tt, npop, tile_base);
                    v[r] = ldcg64(prm.p[i].tmask + (tt - prm.p[i].tile_base));
                }
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const uint32_t tt = t0 + (uint32_t)r * blockDim.x;
                if (tt < TT)
                    tm[tt] = v[r];
            }
        }
        for (uint32_t e = tid; e < kHistSmem; e += blockDim.x)
            bhist[e] = 0u;
        __syncthreads();
        block_scan_chunks_u64(
            TT,
            [&](uint32_t e) {
                const unsigned long long v = tm[e];
                return ((unsigned long long)__popc((uint32_t)v) << 32) | (unsigned long long)__popc((uint32_t)(v >> 32));
            },
            ex, s_tmp64);
        if (tid < npop) {
            const FusedPop &p = prm.p[tid];
            PopSel &s = S[tid];
            const unsigned long long e0 = ex[p.tile_base];
            s.lb = (uint32_t)(e0 >> 32);
            s.eb = (uint32_t)e0;
            const uint32_t last = p.tile_base + p.ntiles - 1u;
            const unsigned long long el = ex[last], vl = tm[last];
            const uint32_t lt_all = (uint32_t)(el >> 32) - s.lb + (uint32_t)__popc((uint32_t)vl);
            const uint32_t eq_all = (uint32_t)el - s.eb + (uint32_t)__popc((uint32_t)(vl >> 32));
            if (lt_all + min(eq_all, s.take) != (uint32_t)(2 * p.N) || s.take > eq_all)
                atomicOr(err, ERR_INTERNAL);
        }
        __syncthreads();
        // m <= 32: two threads per pair
        for (uint32_t w = gwarp; w < nwork_t; w += gwarps) {
            const uint32_t u = w * 32u;
            // the population whose (32-aligned) thread range holds this warp
            int i = -1;
            for (int j = 0; j < npop; ++j)
                if (prm.p[j].m <= 32 && u >= prm.p[j].work_base)
                    i = (i < 0 || prm.p[j].work_base >= prm.p[i].work_base) ? j : i;
            const FusedPop &p = prm.p[i < 0 ? 0 : i];
            const uint32_t local = u + (uint32_t)lane - p.work_base;
            const uint32_t k = local >> 1;
            const int half = (int)(local & 1u);
            const bool valid = i >= 0 && k < (uint32_t)p.N;
            const uint32_t gen = S[i < 0 ? 0 : i].gen0 + 1u + (uint32_t)t;
            Pre pre = pre0;
            if (w != gwarp && valid)
                pre = make_pre(p, gen, (uint32_t)t, k, half);
            uint32_t fpar = 0, spar = 0, fch = 0, sch = 0;
            const PopSel &s = S[i < 0 ? 0 : i];
            switch (p.m) {
#define HADGA_PT(MM)                                                                                        \
    case MM:                                                                                                \
        pair_thread<MM>(p, s, src, gen, pre, k, half, valid, sv, err, fpar, spar, fch, sch);                \
        break;
                HADGA_PT(4) HADGA_PT(8) HADGA_PT(12) HADGA_PT(16) HADGA_PT(20) HADGA_PT(24) HADGA_PT(28) HADGA_PT(32)
#undef HADGA_PT
            default:
                break;
            }
            if (s.boff != 0xFFFFFFFFu) {
                uint32_t *bh = bhist + s.boff;
                if (valid && fpar <= s.capn)
                    atomicAdd(bh + (fpar >> s.shiftn), 1u);
                if (valid && fch <= s.capn)
                    atomicAdd(bh + (fch >> s.shiftn), 1u);
            } else {
                uint32_t *hn = hist_of(p, par ^ 1);
                warp_hist_add(hn, valid && fpar <= s.capn, fpar >> s.shiftn);
                warp_hist_add(hn, valid && fch <= s.capn, fch >> s.shiftn);
            }
            const uint32_t orr = warp_or(valid ? (fpar | fch) : 0u);
            unsigned long long key = ~0ull;
            if (valid) {
                const unsigned long long k1 = ((unsigned long long)fpar << 32) | spar;
                const unsigned long long k2 = ((unsigned long long)fch << 32) | sch;
                key = k1 < k2 ? k1 : k2;
            }
            key = warp_min_u64(key);
            if (lane == 0 && i >= 0) {
                atomicOr(&S[i].bor, orr);
                atomicMin(&S[i].bbest, key);
            }
        }
        // 32 < m <= 128: a warp per pair
        for (uint32_t pr = gwarp; pr < prm.warp_pairs; pr += gwarps) {
            int i = -1;
            for (int j = 0; j < npop; ++j)
                if (prm.p[j].m > 32 && pr >= prm.p[j].work_base && pr < prm.p[j].work_base + (uint32_t)prm.p[j].N)
                    i = j;
            if (i < 0)
                continue;
            const FusedPop &p = prm.p[i];
            const uint32_t k = pr - p.work_base;
            uint32_t *hn = hist_of(p, par ^ 1);
            const uint32_t gen = S[i].gen0 + 1u + (uint32_t)t;
            switch (p.W) {
            case 2: pair_warp<2>(p, S[i], src, gen, (uint32_t)t, k, sv, err, wbuf, hn, bhist); break;
            case 3: pair_warp<3>(p, S[i], src, gen, (uint32_t)t, k, sv, err, wbuf, hn, bhist); break;
            case 4: pair_warp<4>(p, S[i], src, gen, (uint32_t)t, k, sv, err, wbuf, hn, bhist); break;
            default: break;
            }
        }
        // one flush per block of its histogram counts, OR word and best key
        __syncthreads();
        for (int i = 0; i < npop; ++i) {
            const uint32_t bo = S[i].boff;
            if (bo == 0xFFFFFFFFu)
                continue;
            const uint32_t nb = (S[i].capn >> S[i].shiftn) + 1u;
            uint32_t *hn = hist_of(prm.p[i], par ^ 1);
            for (uint32_t e = tid; e < nb; e += blockDim.x) {
                const uint32_t c = bhist[bo + e];
                if (c)
                    atomicAdd(hn + e, c);
            }
        }
        if (tid < npop) {
            const FusedPop &p = prm.p[tid];
            if (S[tid].bor)
                atomicOr(stat_of(p) + 1 + (par ^ 1), S[tid].bor);
            if (S[tid].bbest != ~0ull)
                atomicMin(p.traj + (S[tid].gen0 + (uint32_t)t) % (uint32_t)p.traj_cap, S[tid].bbest);
        }
        if (!grid_barrier(prm.bar, nblocks, epoch, err))
            return;
        src ^= 1;
        if (tid < npop) {
            S[tid].cap = S[tid].capn;
            S[tid].shift = S[tid].shiftn;
        }
        done = t + 1;
        if (prm.stop_at_zero) {
            const FusedPop &p = prm.p[0];
            const unsigned long long key = ldcg64(p.traj + (S[0].gen0 + (uint32_t)t) % (uint32_t)p.traj_cap);
            if ((key >> 32) == 0ull)
                break;
        }
        __syncthreads();
    }
    if (blockIdx.x == 0 && tid == 0)
        *prm.done = done;
    if (blockIdx.x == 0 && tid < npop)
        *prm.p[tid].gen_dev = S[tid].gen0 + (uint32_t)done;
}

size_t fused_smem_bytes(const FusedParams &p)
{
    const size_t r1 = std::max((size_t)4 * p.total_tiles, (size_t)2 * kHistSmem);
    return (r1 + kHistSmem + (size_t)(kFusedThreads / 32) * p.warp_buf_words) * 4u;
}

cudaError_t fused_grid(size_t smem, int *grid)
{
    cudaError_t e = cudaFuncSetAttribute(k_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fused, kFusedThreads, smem);
    if (e != cudaSuccess)
        return e;
    if (per < 1)
        return cudaErrorCooperativeLaunchTooLarge;
    *grid = sms;  // one resident block per SM
    return cudaSuccess;
}

cudaError_t launch_fused(const FusedParams &p, int grid, size_t smem, cudaStream_t s)
{
    void *args[] = {(void *)&p};
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)k_fused, dim3(grid), dim3(kFusedThreads), args, smem, s);
    if (e == cudaSuccess)
        note_launches(1);
    return e;
}

} // namespace hadga
