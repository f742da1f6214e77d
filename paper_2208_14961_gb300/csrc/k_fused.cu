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
//           offspring run in registers (m <= 32: four threads per pair,
//           two per offspring) or in shared memory (32 < m <= 128: a warp
//           per offspring); the new population goes to the other ping-pong buffer and
//           the histogram, OR word and best key of generation g + 1 are
//           accumulated with warp-aggregated atomics.
// Data written inside the launch is read with ld.global.cg (L2) so no SM
// can see a stale L1 line across generations.
#include <algorithm>

#include "common.cuh"
#include "inc_plan.cuh"
#include "kernels.cuh"

namespace hadga {

namespace {

constexpr uint32_t FULL = 0xFFFFFFFFu;

struct PopSel {
    uint32_t cap, shift;  // histogram of the current generation: bucket hkey(f) for f <= cap
    uint32_t hlo, hlon;   // window base of the current / next generation's histogram (0: no window)
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
    uint32_t psel;          // probabilistic selection (no threshold, no histograms)
    unsigned long long pbase, pW;  // probabilistic selection: joint prefix before the first tile, total weight
};

__device__ __forceinline__ uint32_t ldcg32(const uint32_t *p) { return __ldcg(p); }
__device__ __forceinline__ unsigned long long ldcg64(const unsigned long long *p) { return __ldcg(p); }

// smallest s with (cap >> s) < kHistR
__device__ __forceinline__ uint32_t shift_for(uint32_t cap)
{
    const int bl = 32 - __clz(cap);
    return bl > 12 ? (uint32_t)(bl - 12) : 0u;
}

// Histogram bucket of fitness f (f <= cap) with window base lo and bucket
// width 2^sh: values below the window share bucket 0.
__device__ __forceinline__ uint32_t hkey(uint32_t f, uint32_t lo, uint32_t sh)
{
    return f >= lo ? (f - lo) >> sh : 0u;
}

// Buckets of a histogram up to cap.
__device__ __forceinline__ uint32_t hbuckets(uint32_t cap, uint32_t lo, uint32_t sh)
{
    return ((cap - lo) >> sh) + 1u;
}

// Histogram parameters of the next generation from its cap T (the current
// threshold, a multiple of 2^v): buckets of width max(v, shift_for(T))
// from 0 when that width is exact (<= 2^v); otherwise exact buckets of
// width 2^v over the kHistR - 1 values just below T, everything lower in
// bucket 0 (the next threshold usually moves less than the window; when it
// falls below it, the refinement passes find it).
__device__ __forceinline__ void next_hist(uint32_t T, uint32_t v, uint32_t &lo, uint32_t &sh)
{
    sh = max(v, shift_for(T));
    lo = 0u;
    if (sh > v && v < 20u) {
        const uint32_t span = (uint32_t)(kHistR - 1) << v;
        lo = T > span ? T - span : 0u;
        sh = v;
        if (lo == 0u)
            sh = max(v, shift_for(T));
    }
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

// Whole warp, histogram h[0, n) in shared memory (n <= 4096): bucket b where
// the running count first reaches `need` (1 <= need <= total) and the count
// before it.  Two levels: every lane sums a contiguous chunk (visited in a
// lane-rotated order to spread the banks), a warp scan finds the chunk, the
// 32 lanes split that chunk four buckets each and a second scan finds the
// bucket.  Returns false when no bucket reaches `need`.
__device__ bool warp_find_crossing_smem(const uint32_t *h, uint32_t n, uint32_t need, uint32_t &b_out,
                                        uint32_t &before_out)
{
    const int lane = threadIdx.x & 31;
    const uint32_t per = (((n + 31u) >> 5) + 3u) & ~3u;  // chunk length, a multiple of 4 (<= 128)
    const uint32_t lo = (uint32_t)lane * per, rot = (uint32_t)lane % per;
    uint32_t sum = 0;
    for (uint32_t v = 0; v < per; ++v) {
        uint32_t e = v + rot;
        e = e >= per ? e - per : e;
        if (lo + e < n)
            sum += h[lo + e];
    }
    const uint32_t incl = warp_incl_scan(sum, lane), excl = incl - sum;
    const uint32_t bal = __ballot_sync(FULL, excl < need && need <= incl);
    if (bal == 0u)
        return false;
    const int owner = __ffs(bal) - 1;
    const uint32_t olo = (uint32_t)owner * per;
    const uint32_t base = __shfl_sync(FULL, excl, owner);
    // second level: lane l takes buckets olo + 4l .. olo + 4l + 3 of the chunk
    uint32_t c4[4];
    uint32_t s4 = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t e = olo + 4u * (uint32_t)lane + (uint32_t)k;
        c4[k] = (4u * (uint32_t)lane + (uint32_t)k < per && e < n) ? h[e] : 0u;
        s4 += c4[k];
    }
    const uint32_t i2 = warp_incl_scan(s4, lane);
    uint32_t run = base + i2 - s4;
    int hit = -1;
    uint32_t before = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (hit < 0 && run + c4[k] >= need) {
            hit = k;
            before = run;
        }
        run += c4[k];
    }
    const uint32_t bal2 = __ballot_sync(FULL, hit >= 0);
    if (bal2 == 0u)
        return false;
    const int o2 = __ffs(bal2) - 1;
    b_out = olo + 4u * (uint32_t)o2 + (uint32_t)__shfl_sync(FULL, hit, o2);
    before_out = __shfl_sync(FULL, before, o2);
    return true;
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

// Slot drawn by the probabilistic selection for a parent whose draw is u:
// the tile sums' exclusive prefix ex (joint tile space, shared memory) from
// the population's first tile, then the in-tile weight prefixes.
__device__ __forceinline__ uint32_t psel_slot_of(unsigned long long u, const FusedPop &p, const PopSel &S,
                                                 const Surv &sv, uint32_t *err)
{
    const unsigned long long *ex = sv.ex + p.tile_base;
    return psel_lookup(u, [&](uint32_t j) { return ex[j]; }, p.ntiles, S.pbase, S.pW, p.cw, (uint32_t)(4 * p.N),
                       err);
}

// Stream index of the mutation draws of offspring o: o itself, or 2N for
// every offspring under method 1 of Sec. 3.5 (one draw per generation).
__device__ __forceinline__ uint32_t mut_stream(const FusedPop &p, uint32_t o)
{
    return p.shared_mut ? (uint32_t)(2 * p.N) : o;
}

// Draws of one build item that do not depend on the selection: survivor
// number d, cut point c and (for NC = NR = 1) the mutated column and rows.
struct Pre {
    uint32_t d, c, cc, ra, rb;
    unsigned long long u;  // probabilistic selection: the parent's 64-bit draw
};

__device__ __forceinline__ Pre make_pre(const FusedPop &p, uint32_t gen, uint32_t tch, uint32_t k, int half,
                                        bool psel)
{
    const uint32_t N = (uint32_t)p.N;
    Pre r;
    r.d = 0u;
    r.u = 0ull;
    if (psel)
        r.u = psel_draw(p.seed, p.pop_id, gen, k + (half ? N : 0u));
    else
        r.d = __ldg(p.perm + (size_t)tch * 2u * N + k + (half ? N : 0u));
    r.c = (uint32_t)cut_point(p.seed, p.pop_id, gen, k, p.m);
    r.cc = r.ra = r.rb = 0u;
    if (p.NC == 1 && p.NR == 1) {
        const uint4 w = philox_block(p.seed, p.pop_id, OP_MUTATE, gen, mut_stream(p, k + (half ? N : 0u)), 0u, 0u);
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

// Half of the upper-triangle terms of a column set, chosen so that the same
// code on the columns rotated by one (c'[j] = c[(j + 1) mod M]) yields the
// other half: pairs (a, a + s mod M) with a even, 1 <= s < M/2, plus
// (a, a + M/2) with a even and a < M/2 (M is a multiple of 4).
template <int M, int KIND>
__device__ __forceinline__ uint32_t fitness_half_regs(const uint32_t (&c)[M])
{
    uint32_t acc = 0;
#pragma unroll
    for (int a = 0; a < M; a += 2) {
#pragma unroll
        for (int s = 1; s < M / 2; ++s)
            acc += fit_term<KIND>(M - 2 * __popc(c[a] ^ c[(a + s) % M]));
        if (a < M / 2)
            acc += fit_term<KIND>(M - 2 * __popc(c[a] ^ c[a + M / 2]));
    }
    return acc;
}

// ---------------------------------------------------------------------------
// m <= 32, TPP = 4: four threads per pair (lanes 4j .. 4j + 3): `half`
// selects the offspring O_{1 + half} (and the parent P_{1 + half} it carries
// over), `sub` splits its fitness terms; thread sub = 1 places the parent,
// sub = 0 the offspring.  Each thread returns the one (fitness, slot) it
// placed in f_out[0], slot_out[0].
// TPP = 2: two threads per pair (lanes 2j, 2j + 1 = half), each computing
// all fitness terms of its offspring and placing both the parent it
// carries over (f_out[0], slot_out[0]) and the offspring (f_out[1],
// slot_out[1]).  The autotuner picks TPP per order.
// ---------------------------------------------------------------------------
template <int M, int TPP>
__device__ __forceinline__ void pair_thread(const FusedPop &p, const PopSel &S, int src, uint32_t gen, const Pre &pre,
                                            uint32_t k, int half, int sub, bool valid, const Surv &sv, uint32_t *err,
                                            uint32_t (&f_out)[2], uint32_t (&slot_out)[2])
{
    static_assert(TPP == 2 || TPP == 4, "two or four threads per pair");
    const uint32_t N = (uint32_t)p.N;
    uint32_t s_mine = 0;
    if (valid)
        s_mine = S.psel ? psel_slot_of(pre.u, p, S, sv, err) : survivor_of(pre.d, p, S, sv, err);
    const uint32_t s_other = __shfl_xor_sync(FULL, s_mine, TPP == 4 ? 2 : 1);
    const uint32_t *src_pop = p.pop[src];
    uint32_t *dst_pop = p.pop[src ^ 1];
    const uint32_t s1 = half ? s_other : s_mine, s2 = half ? s_mine : s_other;
    uint32_t p1[M], p2[M];
    if (valid) {
        const uint4 *a = reinterpret_cast<const uint4 *>(src_pop + (size_t)s1 * M);
        const uint4 *b = reinterpret_cast<const uint4 *>(src_pop + (size_t)s2 * M);
#pragma unroll
        for (int v = 0; v < M / 4; ++v) {
            const uint4 x = __ldcg(a + v), y = __ldcg(b + v);
            p1[4 * v] = x.x, p1[4 * v + 1] = x.y, p1[4 * v + 2] = x.z, p1[4 * v + 3] = x.w;
            p2[4 * v] = y.x, p2[4 * v + 1] = y.y, p2[4 * v + 2] = y.z, p2[4 * v + 3] = y.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < M; ++j)
            p1[j] = p2[j] = 0u;
    }
    if (valid && (TPP == 2 || sub)) {
        // the parent this half carries over keeps its slot order k / k + N
        f_out[0] = ldcg32(p.fit[src] + s_mine);
        slot_out[0] = half ? k + N : k;
        uint4 *d = reinterpret_cast<uint4 *>(dst_pop + (size_t)slot_out[0] * M);
#pragma unroll
        for (int v = 0; v < M / 4; ++v) {
            const uint32_t *q = half ? p2 : p1;
            d[v] = make_uint4(q[4 * v], q[4 * v + 1], q[4 * v + 2], q[4 * v + 3]);
        }
        p.fit[src ^ 1][slot_out[0]] = f_out[0];
    }
    // crossover (Sec. 3.4): O1 = P1[:, :c] | P2[:, c:], O2 = P2[:, :c] | P1[:, c:]
    const int c = (int)pre.c;
    uint32_t o[M];
#pragma unroll
    for (int j = 0; j < M; ++j)
        o[j] = ((j < c) != (half != 0)) ? p1[j] : p2[j];
    // mutation (Sec. 3.5): columns in order, pairs in order, flip iff different
    {
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
            Draws dr(p.seed, p.pop_id, gen, mut_stream(p, k + (half ? N : 0u)));
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
    // fitness: this thread's half of the terms (columns rotated by one for
    // sub 1), or both halves with two threads per pair
    uint32_t cr[M];
#pragma unroll
    for (int j = 0; j < M; ++j)
        cr[j] = (TPP == 2 || sub) ? o[(j + 1) % M] : o[j];
    uint32_t part;
    switch (p.kind) {
    case FIT_SQ: part = fitness_half_regs<M, FIT_SQ>(cr); break;
    case FIT_ABS: part = fitness_half_regs<M, FIT_ABS>(cr); break;
    default: part = fitness_half_regs<M, FIT_NNZ>(cr); break;
    }
    uint32_t sum;
    if constexpr (TPP == 4) {
        sum = part + __shfl_xor_sync(FULL, part, 1);
    } else {
        switch (p.kind) {
        case FIT_SQ: sum = part + fitness_half_regs<M, FIT_SQ>(o); break;
        case FIT_ABS: sum = part + fitness_half_regs<M, FIT_ABS>(o); break;
        default: sum = part + fitness_half_regs<M, FIT_NNZ>(o); break;
        }
    }
    const uint32_t f = p.kind == FIT_SQ ? fit_finish<FIT_SQ>(sum) : fit_finish<FIT_ABS>(sum);
    const int oi = TPP == 4 ? 0 : 1;  // output entry of the offspring
    if (valid && (TPP == 2 || !sub)) {
        slot_out[oi] = 2u * N + k + (half ? N : 0u);
        uint4 *d = reinterpret_cast<uint4 *>(dst_pop + (size_t)slot_out[oi] * M);
#pragma unroll
        for (int v = 0; v < M / 4; ++v)
            d[v] = make_uint4(o[4 * v], o[4 * v + 1], o[4 * v + 2], o[4 * v + 3]);
        p.fit[src ^ 1][slot_out[oi]] = f;
        f_out[oi] = f;
    }
}

// ---------------------------------------------------------------------------
// a7 -- incremental fitness of one offspring (warp-wide; not in the paper,
// which recomputes G: derived from the fitness of Sec. 3.2 under the
// operators of Sec. 3.4 and 3.5).
//
// Each individual keeps H = G / 2 (int8) in 8 x 8 tiles of the upper
// triangle (common.cuh); a tile row (i, J) is the 8 bytes H[i][8J .. 8J+7].
// The offspring O takes columns [0, c) from parent Pt and [c, m) from Pb,
// then pair flips change the columns of the set M.  A column exchange keeps
// H[:c, :c] of Pt and H[c:, c:] of Pb, and a pair flip in column cc changes
// only row and column cc, so:
//  Phase 1: the tiles wholly inside H[:c, :c] (tile columns J < c/8) are
//           copied from Pt, the tiles wholly inside H[c:, c:] (tile rows
//           8I >= c, one contiguous run) from Pb, through a per-warp ring
//           of 16-byte cp.async copies (four in flight per lane, no
//           registers held); the tile rows i >= c of the tile row cut by c
//           are copied from Pb with 8-byte loads;
//  Phase 2: the remaining tile rows (i < c, 8J + 8 > c) hold the c (m - c)
//           cross entries: computed by popcount from the final columns `bo`,
//           their bytes j < c taken from Pt; work items (i, J) enumerated
//           row-fastest so every lane carries the same number of dot
//           products and the 8 columns of a tile column are broadcast reads;
//  Phase 3: entries of rows and columns of M outside the cross block still
//           hold the parents' values: recomputed from `bo` and stored byte
//           by byte, and the fitness sum corrected by term(new) - term(old),
//           old from the parents' columns.
// The fitness terms of every stored entry come from SIMD byte arithmetic
// (dp4a).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t mut_word(const uint32_t (&mut)[4], int w)
{
    return w == 0 ? mut[0] : w == 1 ? mut[1] : w == 2 ? mut[2] : mut[3];
}

__device__ __forceinline__ uint32_t mut_bit(const uint32_t (&mut)[4], int i)
{
    return (mut_word(mut, i >> 5) >> (i & 31)) & 1u;
}

// Index of tile row (i, J) in 8-byte units: tile t(I, J) holds units 8t .. 8t+7.
__device__ __forceinline__ uint32_t tile_row_unit(int i, int J, int nb)
{
    const int I = i >> 3;
    return (uint32_t)((I * nb - (I * (I - 1)) / 2 + (J - I)) * 8 + (i & 7));
}

// Issues the cp.async copies of phase-1 groups [base, base + ring) into the
// warp's ring (slot e - base); each lane copies the groups e = lane mod 32.
// With base 0 and the whole plan within the ring, the extra groups follow
// (slots nG ..).
__device__ __forceinline__ void inc_copy_issue(const IncCopyPlan &pl, const int8_t *gt8, const int8_t *gb8,
                                               uint4 *ring, int ring_groups, int base, int lane)
{
    const int end = min(base + ring_groups, pl.nG);
    for (IncGroupIter it(pl, base + lane); it.e < end; it.next(pl))
        cp_async16(ring + (it.e - base), (it.from_pt(pl) ? gt8 : gb8) + (size_t)it.unit(pl) * 16u);
    if (base == 0 && pl.total <= ring_groups) {
        for (int x = lane; x < pl.n4g + pl.n3g; x += 32) {
            bool pt;
            const uint32_t u = pl.extra_unit(x, pt);
            cp_async16(ring + pl.nG + x, (pt ? gt8 : gb8) + (size_t)u * 16u);
        }
    }
}

// The whole copy plan as bulk asynchronous copies (cp.async.bulk, the TMA
// engine's linear form) completing on the warp's mbarrier `bar`: one copy
// per run of consecutive ring slots -- each H[:c, :c] tile row of Pt, the
// H[c:, c:] tiles of Pb, and when 8 does not divide c one per tile of the
// cut tile column (Pt) and of the cut tile row (Pb).  Lane 0 posts the byte
// count first; the lanes then issue the runs r = lane, lane + 32, ...  Only
// when the whole plan fits the ring (pl.total <= ring_groups).
__device__ __forceinline__ void inc_bulk_issue(const IncCopyPlan &pl, const int8_t *gt8, const int8_t *gb8,
                                               uint4 *ring, uint64_t *bar, int lane)
{
    const int nt = pl.nb * (pl.nb + 1) / 2, I0 = pl.J0, nbr = nt > pl.tBR ? 1 : 0;
    const int n4 = pl.r0 ? I0 + 1 : 0, n3 = pl.r0 ? pl.nb - I0 : 0;
    const int nruns = pl.J0 + nbr + n4 + n3;
    // the parents' tiles were written by generic stores before the last grid
    // barrier, and the ring was last read by generic loads: order both
    // before this thread's async copies
    asm volatile("fence.proxy.async.global;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (lane == 0)
        mbar_expect_tx(bar, (uint32_t)pl.total * 16u);
    __syncwarp();
    for (int r = lane; r < nruns; r += 32) {
        const int8_t *src;
        int slot, bytes;
        if (r < pl.J0) {  // tile row I = r of the H[:c, :c] triangle
            const int I = r;
            src = gt8 + 64u * pl.tile(I, I);
            slot = 4 * (I * pl.J0 - (I * (I - 1)) / 2);
            bytes = 64 * (pl.J0 - I);
        } else if (r < pl.J0 + nbr) {
            src = gb8 + 64u * (uint32_t)pl.tBR;
            slot = 4 * pl.nTL;
            bytes = 64 * (nt - pl.tBR);
        } else if (r < pl.J0 + nbr + n4) {  // Pt's rows i < c of tile (I, J0)
            const int I = r - pl.J0 - nbr;
            src = gt8 + 64u * pl.tile(I, pl.J0);
            slot = pl.nG + 4 * I;
            bytes = 16 * (I < I0 ? 4 : (pl.r0 + 1) >> 1);
        } else {  // Pb's rows i >= c of tile (I0, J)
            const int J = I0 + (r - pl.J0 - nbr - n4);
            src = gb8 + 64u * pl.tile(I0, J) + 16u * (uint32_t)(pl.r0 >> 1);
            slot = pl.nG + pl.n4g + (J - pl.J0) * pl.g3;
            bytes = 16 * pl.g3;
        }
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         smem_u32(ring + slot)),
                     "l"(src), "r"(bytes), "r"(smem_u32(bar))
                     : "memory");
    }
}

// The caller has issued the first ring-full of phase-1 copies
// (inc_copy_issue with base 0) before the parent loads, crossover and
// mutation, whose latency the copies overlap.
template <int W, int KIND>
__device__ uint32_t offspring_incremental(const FusedPop &p, const uint32_t *bo, const uint32_t *bt,
                                          const uint32_t *bb, const uint32_t (&mut)[4], int c, uint32_t gt,
                                          uint32_t gbm, uint32_t go, uint4 *ring, int ring_groups, uint64_t *bar,
                                          uint32_t &bar_parity, uint32_t *err, int lane)
{
    const int m = p.m, nb = gram_tiles_nb(m), hm = m >> 1;
    const int8_t *gt8 = p.gram + (size_t)gt * p.dpad, *gb8 = p.gram + (size_t)gbm * p.dpad;
    const uint2 *Gt = reinterpret_cast<const uint2 *>(gt8), *Gb = reinterpret_cast<const uint2 *>(gb8);
    uint2 *Go = reinterpret_cast<uint2 *>(p.gram + (size_t)go * p.dpad);
    uint32_t acc = 0;

    // ---- phase 1: whole tiles of H[:c, :c] (tile columns J < J0) and of
    // H[c:, c:] (tiles t >= tBR), one ring-full at a time
    const IncCopyPlan pl(m, c);
    const int J0 = pl.J0;
    // the extra groups sit in the ring when the whole plan fit (8-byte rows)
    const bool pre = pl.total <= ring_groups;
    if (pre) {
        // one bulk-copy phase of the warp's mbarrier (bounded wait)
        mbar_wait(bar, bar_parity, err);
        bar_parity ^= 1u;
    }
    for (int base = 0; base < pl.nG; base += ring_groups) {
        if (base > 0)
            inc_copy_issue(pl, gt8, gb8, ring, ring_groups, base, lane);
        if (!pre)
            cp_async_wait_all();
        const int end = min(base + ring_groups, pl.nG);
        for (IncGroupIter it(pl, base + lane); it.e < end; it.next(pl)) {
            const uint4 v = ring[it.e - base];
            __stcg(reinterpret_cast<uint4 *>(Go) + it.unit(pl), v);
            acc += (uint32_t)(word_terms<KIND>(v.x) + word_terms<KIND>(v.y) + word_terms<KIND>(v.z) +
                              word_terms<KIND>(v.w));
        }
        if (base + ring_groups < pl.nG)
            __syncwarp();  // the ring is refilled by other lanes' copies next round
    }
    const uint2 *ring8 = reinterpret_cast<const uint2 *>(ring) + 2 * pl.nG;
    // tile rows i >= c of the tile row I0 = c / 8 cut by c (from Pb)
    if (c & 7) {
        const int I0 = c >> 3, r0 = c & 7, nr = 8 - r0, tot = nr * (nb - I0);
        for (int e = lane; e < tot; e += 32) {
            const int J = I0 + e / nr, i = 8 * I0 + r0 + e % nr;
            const uint32_t un = tile_row_unit(i, J, nb);
            const uint2 v = pre ? ring8[2 * (pl.n4g + (J - J0) * pl.g3 + ((i & 7) >> 1) - (r0 >> 1)) + (i & 1)]
                                : __ldcg(Gb + un);
            __stcg(Go + un, v);
            acc += (uint32_t)(word_terms<KIND>(v.x) + word_terms<KIND>(v.y));
        }
    }

    // ---- phase 2: tile rows (i, J), i < c, J >= J0; item e = (J - J0) c + i
    {
        const int total = c * (nb - J0);
        int i = lane % c, J = J0 + lane / c;
        for (int e = lane; e < total; e += 32) {
            const int j0 = 8 * J;
            const uint32_t un = tile_row_unit(i, J, nb);
            uint2 x = j0 < c ? (pre ? ring8[i] : __ldcg(Gt + un)) : make_uint2(0u, 0u);
            uint32_t ci[W];
            load_col<W>(bo + i * W, ci);
            // the eight dot products are computed unconditionally (column
            // index clamped into the matrix) so their loads issue together;
            // the bytes j < c or j >= m keep the parent's value
#pragma unroll
            for (int hw = 0; hw < 2; ++hw) {
                uint32_t xw = hw ? x.y : x.x;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int j = j0 + 4 * hw + k;
                    uint32_t cj[W];
                    load_col<W>(bo + min(j, m - 1) * W, cj);
                    const uint32_t h = (uint32_t)(hm - xor_popc<W>(ci, cj)) & 0xFFu;
                    const uint32_t keep = (j >= c && j < m) ? ~(0xFFu << (8 * k)) : 0xFFFFFFFFu;
                    xw = (xw & keep) | (h << (8 * k) & ~keep);
                }
                if (hw)
                    x.y = xw;
                else
                    x.x = xw;
            }
            __stcg(Go + un, x);
            acc += (uint32_t)(word_terms<KIND>(x.x) + word_terms<KIND>(x.y));
            i += 32;
            while (i >= c) {
                i -= c;
                ++J;
            }
        }
    }

    // ---- phase 3: rows and columns of the flipped columns, outside the
    // cross block (which phase 2 computed from the final columns)
    if ((mut[0] | mut[1] | mut[2] | mut[3]) != 0u) {
        __syncwarp();
        int8_t *Gob = reinterpret_cast<int8_t *>(Go);
        // column x before the mutation: the parent column at its place
        auto old_col = [&](int x) { return (x < c ? bt : bb) + x * W; };
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            uint32_t bits = mut[w];
            while (bits) {
                const int cc = 32 * w + __ffs(bits) - 1;
                bits &= bits - 1u;
                uint32_t cn[W], co[W];
                load_col<W>(bo + cc * W, cn);
                load_col<W>(old_col(cc), co);
                // column cc: entries (i, cc), i < cc (rows of M included)
                for (int i = lane; i < cc; i += 32) {
                    if (i < c && cc >= c)
                        continue;  // a cross entry
                    uint32_t xn[W], xo[W];
                    load_col<W>(bo + i * W, xn);
                    load_col<W>(mut_bit(mut, i) ? old_col(i) : bo + i * W, xo);
                    const uint32_t hn = (uint32_t)(hm - xor_popc<W>(xn, cn)) & 0xFFu;
                    const uint32_t ho = (uint32_t)(hm - xor_popc<W>(xo, co)) & 0xFFu;
                    __stcg(Gob + (size_t)tile_row_unit(i, cc >> 3, nb) * 8u + (cc & 7), (int8_t)hn);
                    acc += (uint32_t)(word_terms<KIND>(hn) - word_terms<KIND>(ho));
                }
                // row cc: entries (cc, j), j > cc, j not in M (those are
                // handled by column j's pass)
                for (int j = cc + 1 + lane; j < m; j += 32) {
                    if (mut_bit(mut, j) || (cc < c && j >= c))
                        continue;
                    uint32_t xj[W];
                    load_col<W>(bo + j * W, xj);
                    const uint32_t hn = (uint32_t)(hm - xor_popc<W>(cn, xj)) & 0xFFu;
                    const uint32_t ho = (uint32_t)(hm - xor_popc<W>(co, xj)) & 0xFFu;
                    __stcg(Gob + (size_t)tile_row_unit(cc, j >> 3, nb) * 8u + (j & 7), (int8_t)hn);
                    acc += (uint32_t)(word_terms<KIND>(hn) - word_terms<KIND>(ho));
                }
            }
        }
    }
    return word_terms_finish<KIND>(warp_sum(acc));
}

// ---------------------------------------------------------------------------
// 32 < m <= 128: a warp per offspring, matrices staged in shared memory.
// ---------------------------------------------------------------------------
template <int W, bool INC>
__device__ void offspring_warp(const FusedPop &p, PopSel &S, int src, uint32_t gen, uint32_t tch, uint32_t k,
                               int half, const Surv &sv, uint32_t *err, uint32_t *buf, uint4 *ring,
                               int ring_groups, uint64_t *bar, uint32_t &bar_parity, uint32_t *hist_next,
                               uint32_t *bhist)
{
    const int lane = threadIdx.x & 31;
    const int m = p.m;
    const uint32_t N = (uint32_t)p.N, words = (uint32_t)(m * W);
    const uint32_t oh = half ? N : 0u;  // slot offset of this half: parent k + oh, offspring 2N + k + oh
    const bool inc = INC && p.gram != nullptr;
    const int c = cut_point(p.seed, p.pop_id, gen, k, m);
    // lanes 0, 1: slots of the parents (survivors pi(k), pi(k + N)) and
    // their fitness; lane 2 (incremental mode): slot of non-survivor k + oh,
    // whose Gram buffer the offspring takes over
    uint32_t look = 0, lf = 0, lg = 0;
    if (lane < (inc ? 3 : 2)) {
        if (lane < 2)
            look = S.psel ? psel_slot_of(psel_draw(p.seed, p.pop_id, gen, k + (lane ? N : 0u)), p, S, sv, err)
                          : survivor_of(__ldg(p.perm + (size_t)tch * 2u * N + k + (lane ? N : 0u)), p, S, sv, err);
        else
            look = nonsurvivor_of(k + oh, p, S, sv, err);
        // fitness and Gram index of the slot in one round trip
        if (lane < 2)
            lf = ldcg32(p.fit[src] + look);
        if (inc)
            lg = ldcg32(p.gidx[src] + look);
    }
    const uint32_t s1 = __shfl_sync(FULL, look, 0), s2 = __shfl_sync(FULL, look, 1);
    uint32_t *b1 = buf, *b2 = buf + words, *bo = buf + 2 * words;
    const uint32_t *sp = p.pop[src];
    uint32_t *dp = p.pop[src ^ 1];
    const uint32_t w4 = words >> 2;  // words is a multiple of 4
    // the parent giving columns [0, c) (the one this half carries over) and
    // the one giving [c, m)
    const uint32_t st = half ? s2 : s1, sb = half ? s1 : s2;
    const uint4 *pt = reinterpret_cast<const uint4 *>(sp) + (size_t)st * w4;
    const uint4 *pb = reinterpret_cast<const uint4 *>(sp) + (size_t)sb * w4;
    if (inc) {
        // both parents as 16-byte cp.async copies (one commit group, waited
        // for below while the incremental Gram copies stay in flight)
        for (uint32_t e = lane; e < w4; e += 32) {
            cp_async16(reinterpret_cast<uint4 *>(half ? b2 : b1) + e, pt + e);
            cp_async16(reinterpret_cast<uint4 *>(half ? b1 : b2) + e, pb + e);
        }
    } else {
        // full recomputation: the carried-over parent into b1, and the
        // offspring's column set assembled by the copies themselves (Sec. 3.4:
        // columns [0, c) of P_t, [c, m) of P_b, then again columns
        // 0 .. m/2 - 2 for the warp-level Gram).  A 16-byte unit holds words
        // of at most two columns (W >= 2): the one source unit g that the cut
        // splits (its copies in both runs) is merged from both parents through
        // registers by every lane that meets it.
        const uint32_t ext = (uint32_t)(((m >> 1) - 1) * W);
        const uint32_t units = (words + ext + 3u) >> 2;
        uint32_t split = 0xFFFFFFFFu;  // the source unit cut by c, when this lane meets it
        for (uint32_t e = lane; e < w4; e += 32)
            cp_async16(reinterpret_cast<uint4 *>(b1) + e, pt + e);
        for (uint32_t u = lane; u < units; u += 32) {
            const uint32_t g = u < w4 ? u : u - w4;  // unit of the source matrix
            const int j0 = (int)(4u * g) / W, j1 = (int)(4u * g + 3u) / W;
            if (j1 < c)
                cp_async16(reinterpret_cast<uint4 *>(bo) + u, pt + g);
            else if (j0 >= c)
                cp_async16(reinterpret_cast<uint4 *>(bo) + u, pb + g);
            else
                split = g;
        }
        if (split != 0xFFFFFFFFu) {
            // word-wise merge of the cut unit (read through L2, like the copies)
            const uint4 a = __ldcg(pt + split), b = __ldcg(pb + split);
            const uint32_t wa[4] = {a.x, a.y, a.z, a.w}, wb[4] = {b.x, b.y, b.z, b.w};
            uint32_t o[4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
                o[i] = ((int)(4u * split + (uint32_t)i) / W < c) ? wa[i] : wb[i];
            const uint4 v = make_uint4(o[0], o[1], o[2], o[3]);
            reinterpret_cast<uint4 *>(bo)[split] = v;
            if (w4 + split < units)
                reinterpret_cast<uint4 *>(bo)[w4 + split] = v;
        }
    }
    cp_async_commit();
    const uint32_t Fp = __shfl_sync(FULL, lf, half);  // fitness of the parent this half carries over
    // incremental mode: parents keep their Gram buffers, offspring take the
    // buffers of the non-survivors
    uint32_t gb1 = 0, gb2 = 0, go = 0;
    bool gram_group = false;  // the Gram tiles travel as a cp.async group (plan larger than the ring)
    if (inc) {
        const uint32_t P = (uint32_t)(4 * p.N);
        uint32_t g = lg;
        if (g >= P) {
            atomicOr(err, ERR_INTERNAL);  // never expected: indices stay a permutation of [0, P)
            g = 0u;
        }
        if (lane == half)
            p.gidx[src ^ 1][k + oh] = g;
        if (lane == 2)
            p.gidx[src ^ 1][2u * N + k + oh] = g;
        gb1 = __shfl_sync(FULL, g, 0);
        gb2 = __shfl_sync(FULL, g, 1);
        go = __shfl_sync(FULL, g, 2);
        // the parents' Gram tiles start moving now, under the parent loads,
        // crossover and mutation below
        if constexpr (INC) {
            const IncCopyPlan pl(m, c);
            const int8_t *gt8 = p.gram + (size_t)(half ? gb2 : gb1) * p.dpad;
            const int8_t *gb8 = p.gram + (size_t)(half ? gb1 : gb2) * p.dpad;
            if (pl.total <= ring_groups) {
                inc_bulk_issue(pl, gt8, gb8, ring, bar, lane);
            } else {
                inc_copy_issue(pl, gt8, gb8, ring, ring_groups, 0, lane);
                cp_async_commit();
                gram_group = true;
            }
        }
    }
    // mutation draws (Sec. 3.5) in lane 0, while the parents are in flight
    uint8_t cols[64], r1[64], r2[64];
    if (lane == 0) {
        Draws dr(p.seed, p.pop_id, gen, mut_stream(p, k + oh));
        for (int jc = 0; jc < p.NC; ++jc)
            cols[jc] = (uint8_t)uniform_int(dr.next(), 1u, (uint32_t)(m - 1));
        for (int ir = 0; ir < p.NR; ++ir)
            r1[ir] = (uint8_t)uniform_int(dr.next(), 0u, (uint32_t)(m - 1));
        for (int ir = 0; ir < p.NR; ++ir)
            r2[ir] = (uint8_t)uniform_int(dr.next(), 0u, (uint32_t)(m - 1));
    }
    // the parents have landed once at most the Gram group (if any) is pending
    if (gram_group)
        cp_async_wait_group<1>();
    else
        cp_async_wait_group<0>();
    __syncwarp();
    {
        // this half's parent keeps its place k + oh in the next population
        const uint4 *bp = reinterpret_cast<const uint4 *>(inc && half ? b2 : b1);
        uint4 *d4 = reinterpret_cast<uint4 *>(dp) + (size_t)(k + oh) * w4;
        for (uint32_t e = lane; e < w4; e += 32)
            d4[e] = bp[e];
    }
    if (lane == 0)
        p.fit[src ^ 1][k + oh] = Fp;
    // crossover (Sec. 3.4): O1 = P1[:, :c] | P2[:, c:], O2 = P2[:, :c] | P1[:, c:]
    // (full recomputation: already assembled by the copies)
    if (inc) {
        for (uint32_t e = lane; e < words; e += 32)
            bo[e] = (((int)(e / W) < c) != (half != 0)) ? b1[e] : b2[e];
        __syncwarp();
    }
    // mutation (Sec. 3.5) in lane 0, sequential semantics; mut marks the
    // columns where a flip happened
    uint32_t mut[4] = {0u, 0u, 0u, 0u};
    if (lane == 0) {
        for (int jc = 0; jc < p.NC; ++jc) {
            const int cc = cols[jc];
            uint32_t *col = bo + cc * W;
            // full recomputation: the copy of column cc after column m - 1
            // (columns 0 .. m/2 - 2) takes the same flips
            uint32_t *mir = (!inc && cc < (m >> 1) - 1) ? bo + (m + cc) * W : nullptr;
            for (int ir = 0; ir < p.NR; ++ir) {
                const int ra = r1[ir], rb = r2[ir];
                const uint32_t ba = (col[ra >> 5] >> (ra & 31)) & 1u, bb = (col[rb >> 5] >> (rb & 31)) & 1u;
                if (ba != bb) {
                    col[ra >> 5] ^= 1u << (ra & 31);
                    col[rb >> 5] ^= 1u << (rb & 31);
                    if (mir) {
                        mir[ra >> 5] ^= 1u << (ra & 31);
                        mir[rb >> 5] ^= 1u << (rb & 31);
                    }
                    mut[cc >> 5] |= 1u << (cc & 31);
                }
            }
        }
    }
    __syncwarp();
    uint32_t f = 0;
    if constexpr (INC) {
        if (inc) {
#pragma unroll
            for (int w = 0; w < 4; ++w)
                mut[w] = __shfl_sync(FULL, mut[w], 0);
            const uint32_t gt = half ? gb2 : gb1, gbm = half ? gb1 : gb2;
            const uint32_t *bt = half ? b2 : b1, *bb = half ? b1 : b2;  // parents giving [0, c) and [c, m)
            switch (p.kind) {
            case FIT_SQ: f = offspring_incremental<W, FIT_SQ>(p, bo, bt, bb, mut, c, gt, gbm, go, ring, ring_groups, bar, bar_parity, err, lane); break;
            case FIT_ABS: f = offspring_incremental<W, FIT_ABS>(p, bo, bt, bb, mut, c, gt, gbm, go, ring, ring_groups, bar, bar_parity, err, lane); break;
            default: f = offspring_incremental<W, FIT_NNZ>(p, bo, bt, bb, mut, c, gt, gbm, go, ring, ring_groups, bar, bar_parity, err, lane); break;
            }
        }
    }
    if (!inc) {
        // the warp-level Gram reads the copies of columns 0 .. m/2 - 2 after
        // column m - 1 (made by the copies and the mutation above)
        switch (p.kind) {
        case FIT_SQ: f = warp_fitness_cols<W, FIT_SQ>(bo, m, lane, p.nch); break;
        case FIT_ABS: f = warp_fitness_cols<W, FIT_ABS>(bo, m, lane, p.nch); break;
        default: f = warp_fitness_cols<W, FIT_NNZ>(bo, m, lane, p.nch); break;
        }
    }
    const uint32_t slot = 2u * N + k + oh;
    for (uint32_t e = lane; e < (words >> 2); e += 32)
        reinterpret_cast<uint4 *>(dp)[(size_t)slot * (words >> 2) + e] = reinterpret_cast<const uint4 *>(bo)[e];
    if (lane == 0) {
        p.fit[src ^ 1][slot] = f;
        const uint32_t fv[2] = {Fp, f};
        const uint32_t slots[2] = {k + oh, slot};
        unsigned long long bk = ~0ull;
        uint32_t orr = 0;
        for (int i = 0; i < 2; ++i) {
            if (!S.psel && fv[i] <= S.capn)
                atomicAdd((S.boff != 0xFFFFFFFFu ? bhist + S.boff : hist_next) + hkey(fv[i], S.hlon, S.shiftn), 1u);
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

// INC: compiled with the incremental Gram path of the warp-per-pair build
// (launched when a population keeps its Gram), so that its register needs
// stay out of the other instantiation.
template <bool INC>
__global__ void __launch_bounds__(kFusedThreads, 1) k_fused(const __grid_constant__ FusedParams prm)
{
    extern __shared__ __align__(16) uint32_t dyn[];
    __shared__ PopSel S[kMaxPops];
    // the populations' parameters, copied once from the kernel argument: read
    // with population indices computed at run time, the argument would be
    // served by the constant cache, whose misses cost L2 round trips on the
    // dependent chains of the build phase
    __shared__ __align__(16) FusedPop PP[kMaxPops];
    __shared__ unsigned long long s_tmp64[32];
    __shared__ uint32_t hoff[kMaxPops];
    __shared__ int s_flag;
    __shared__ uint32_t s_next;  // next warp item of the block (phase B)
    __shared__ __align__(8) uint64_t s_incbar[kFusedThreads / 32];  // per-warp bulk-copy barrier

    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    const int npop = prm.npop;
    {
        static_assert(sizeof(FusedPop) % 4 == 0, "FusedPop copies word by word");
        const uint32_t *from = reinterpret_cast<const uint32_t *>(prm.p);
        uint32_t *to = reinterpret_cast<uint32_t *>(PP);
        for (uint32_t e = tid; e < (uint32_t)npop * (uint32_t)(sizeof(FusedPop) / 4); e += blockDim.x)
            to[e] = from[e];
        __syncthreads();
    }
    const uint32_t nblocks = gridDim.x;
    const uint32_t gtid = blockIdx.x * blockDim.x + tid, gthreads = nblocks * blockDim.x;
    // warps enumerated across blocks first, so consecutive work items land on
    // different SMs
    const uint32_t gwarp = (uint32_t)wib * nblocks + blockIdx.x, gwarps = gthreads >> 5;
    const uint32_t TT = prm.total_tiles;
    // [tile masks and their prefix (phase B) | incremental copy ring (phase B)
    //  | staged histograms (phase A, overlapping both)] [bhist] [warp buffers]
    const uint32_t ring_words = INC ? (uint32_t)(kFusedThreads / 32) * (uint32_t)prm.inc_ring * 4u : 0u;
    const uint32_t r1 = max(4u * TT + ring_words, 2u * kHistSmem);
    unsigned long long *tm = reinterpret_cast<unsigned long long *>(dyn);
    unsigned long long *ex = tm + TT;
    uint32_t *hcnt = dyn;
    uint4 *ring = reinterpret_cast<uint4 *>(dyn + 4u * TT) + wib * prm.inc_ring;
    uint32_t *bhist = dyn + r1;  // block-local histograms of the next generation
    uint32_t *wbuf = bhist + kHistSmem + wib * prm.warp_buf_words;
    const Surv sv{tm, ex};
    uint32_t *err = prm.err;
    uint32_t epoch = 0;
    uint32_t inc_parity = 0;  // phase of this warp's bulk-copy barrier
    if (INC && tid < kFusedThreads / 32) {
        mbar_init(&s_incbar[tid], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    int src = prm.src;
    int done = 0;
    auto tile_base = [&](int i) { return PP[i].tile_base; };

    // ---- pre-pass: max and OR of the current fitness of every population -----
    // (truncation selection only: probabilistic selection keeps no histograms)
    const bool psel = prm.psel != 0;
    if (tid < npop) {
        S[tid].gen0 = ldcg32(PP[tid].gen_dev);
        S[tid].psel = psel ? 1u : 0u;
        S[tid].boff = 0xFFFFFFFFu;
        S[tid].hlo = 0u;  // the launch's first histogram covers [0, max F] from bucket 0
    }
    __syncthreads();
    if (!psel) {
        const int par0 = 0;  // buffers alternate with the generation index inside the launch
        for (int i = 0; i < npop; ++i) {
            const FusedPop &p = PP[i];
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
            const FusedPop &p = PP[tid];
            const uint32_t cap = ldcg32(stat_of(p) + 0);
            const uint32_t v = ctz_or(ldcg32(stat_of(p) + 1 + par0));
            S[tid].cap = cap;
            S[tid].shift = max(v, shift_for(cap));
        }
        __syncthreads();
        for (int i = 0; i < npop; ++i) {
            const FusedPop &p = PP[i];
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

    // the selection-independent draws (survivor number or parent draw, cut
    // point, mutation) of this thread's first m <= 32 build item of
    // generation tt of the launch
    auto first_pre = [&](int tt) {
        Pre r{0u, 1u, 1u, 0u, 0u, 0ull};
        const uint32_t u = gwarp * 32u + (uint32_t)lane;
        if (gwarp < (prm.thread_slots >> 5)) {
            int i = -1;
            for (int j = 0; j < npop; ++j)
                if (PP[j].m <= 32 && u >= PP[j].work_base)
                    i = (i < 0 || PP[j].work_base >= PP[i].work_base) ? j : i;
            if (i >= 0) {
                const FusedPop &p = PP[i];
                const uint32_t local = u - p.work_base;
                const uint32_t k = p.tpp == 2 ? local >> 1 : local >> 2;
                const int half = (int)(p.tpp == 2 ? (local & 1u) : ((local >> 1) & 1u));
                if (k < (uint32_t)p.N)
                    r = make_pre(p, S[i].gen0 + 1u + (uint32_t)tt, (uint32_t)tt, k, half, psel);
            }
        }
        return r;
    };
    Pre pre_next{0u, 1u, 1u, 0u, 0u, 0ull};
    uint32_t ref_level = 0;
    for (int t = 0; t < prm.ngen; ++t) {
        const int par = t & 1;

        // ---- phase A: threshold of the 2N smallest ---------------------------------
        // loads first: the OR word of the current fitness values and the
        // first group's histogram buckets (populations [0, g1) whose buckets
        // fit the staging area), held in registers while the
        // selection-independent draws are computed
        const uint32_t vload = (!psel && tid < npop) ? ldcg32(stat_of(PP[tid]) + 1 + par) : 0u;
        int g1 = 0;
        uint32_t goff = 0;
        while (!psel && g1 < npop) {
            const uint32_t nb = hbuckets(S[g1].cap, S[g1].hlo, S[g1].shift);
            if (g1 > 0 && goff + nb > kHistSmem)
                break;
            goff += nb;
            ++g1;
        }
        constexpr int kStageRegs = 8;  // buckets per thread staged through registers
        uint32_t hv[kStageRegs];
#pragma unroll
        for (int r = 0; r < kStageRegs; ++r) {
            const uint32_t e = (uint32_t)tid + (uint32_t)r * kFusedThreads;
            hv[r] = 0u;
            if (e < goff) {
                int i = 0;
                uint32_t base = 0, nb = hbuckets(S[0].cap, S[0].hlo, S[0].shift);
                while (i + 1 < g1 && e >= base + nb) {
                    base += nb;
                    ++i;
                    nb = hbuckets(S[i].cap, S[i].hlo, S[i].shift);
                }
                hv[r] = ldcg32(hist_of(PP[i], par) + (e - base));
            }
        }
        // first tile of this warp: its fitness is loaded now, with the histograms
        uint32_t f_pre = 0;
        int i_pre = 0;
        if (gwarp < TT) {
            i_pre = owner_of(gwarp, npop, tile_base);
            const FusedPop &p = PP[i_pre];
            const uint32_t q = (gwarp - p.tile_base) * 32u + lane;
            f_pre = q < (uint32_t)(4 * p.N) ? ldcg32(p.fit[src] + q) : 0u;
        }
        // selection-independent draws of this warp's first build item: drawn
        // while the previous generation's closing barrier completed, except in
        // the launch's first generation
        const uint32_t nwork_t = prm.thread_slots >> 5;
        const Pre pre0 = t == 0 ? first_pre(0) : pre_next;
        for (int i = 0; i < npop && !psel; ++i) {
            uint32_t *hn = hist_of(PP[i], par ^ 1);
            for (uint32_t e = gtid; e < (uint32_t)kHistR; e += gthreads)
                hn[e] = 0u;
        }
        if (blockIdx.x == 0 && tid < npop) {
            const FusedPop &p = PP[tid];
            stat_of(p)[1 + (par ^ 1)] = 0u;
            p.traj[(S[tid].gen0 + (uint32_t)t) % (uint32_t)p.traj_cap] = ~0ull;
        }
        if (tid == 0)
            s_flag = 0;
        // histograms staged in shared memory (groups of populations that
        // fit); one warp per population finds the crossing of 2N and, when
        // its bucket holds a single value, fixes the threshold right away
        for (int i0 = 0; i0 < npop && !psel;) {
            uint32_t off = 0;
            int i1 = i0;
            while (i1 < npop) {
                const uint32_t nb = hbuckets(S[i1].cap, S[i1].hlo, S[i1].shift);
                if (i1 > i0 && off + nb > kHistSmem)
                    break;
                if (tid == 0)
                    hoff[i1] = off;
                off += nb;
                ++i1;
            }
            if (i0 == 0) {
                // the first group: from the registers, and beyond them directly
#pragma unroll
                for (int r = 0; r < kStageRegs; ++r) {
                    const uint32_t e = (uint32_t)tid + (uint32_t)r * kFusedThreads;
                    if (e < off)
                        hcnt[e] = hv[r];
                }
                if (tid < npop) {
                    S[tid].v = ctz_or(vload);
                    S[tid].need = 0xFFFFFFFFu;  // marks "crossing not found"
                }
                __syncthreads();
                for (uint32_t e = (uint32_t)tid + kStageRegs * kFusedThreads; e < off; e += blockDim.x) {
                    int i = 0;
                    while (i + 1 < i1 && e >= hoff[i + 1])
                        ++i;
                    hcnt[e] = ldcg32(hist_of(PP[i], par) + (e - hoff[i]));
                }
            } else {
                __syncthreads();
                for (uint32_t e = tid; e < off; e += blockDim.x) {
                    int i = i0;
                    while (i + 1 < i1 && e >= hoff[i + 1])
                        ++i;
                    hcnt[e] = ldcg32(hist_of(PP[i], par) + (e - hoff[i]));
                }
            }
            __syncthreads();
            if (wib < i1 - i0) {
                const int i = i0 + wib;
                PopSel &s = S[i];
                const uint32_t nb = hbuckets(s.cap, s.hlo, s.shift);
                const uint32_t need2 = (uint32_t)(2 * PP[i].N);
                uint32_t b = 0, before = 0;
                const bool found = warp_find_crossing_smem(hcnt + hoff[i], nb, need2, b, before);
                if (lane == 0) {
                    if (found) {
                        s.lo = s.hlo + (b << s.shift);
                        s.need = need2 - before;
                    } else {
                        atomicOr(err, ERR_INTERNAL);
                        s.lo = 0;
                        s.need = 1;
                    }
                    s.sr = s.shift;
                    s.exact = s.shift <= s.v ? 1u : 0u;
                    if (found && b == 0u && s.hlo != 0u) {
                        // the threshold lies below the window: bucket 0 holds [0, hlo + 2^shift)
                        s.lo = 0u;
                        s.sr = 32u - (uint32_t)__clz(s.hlo + (1u << s.shift) - 1u);
                        s.exact = 0u;
                    }
                    if (s.exact) {
                        s.T = s.lo;
                        s.take = s.need;
                        s.capn = s.T;
                        next_hist(s.T, s.v, s.hlon, s.shiftn);
                        s.bor = 0u;
                        s.bbest = ~0ull;
                    } else {
                        atomicOr(&s_flag, 1);
                    }
                }
            }
            __syncthreads();
            i0 = i1;
        }
        // refinement passes while a candidate bucket may hold several values
        // (s_flag was last written before a block barrier of the staging loop,
        // which probabilistic selection skips: it never reads it)
        if (!psel && s_flag) {
            while (s_flag) {
                const int rl = (int)(ref_level % 3u), rz = (int)((ref_level + 1u) % 3u);
                for (int i = 0; i < npop; ++i) {
                    const FusedPop &p = PP[i];
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
                    const FusedPop &p = PP[wib];
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
                next_hist(s.T, s.v, s.hlon, s.shiftn);
                s.bor = 0u;
                s.bbest = ~0ull;
            }
            __syncthreads();
        }
        // tile masks: F < T and F == T per 32 slots
        for (uint32_t tl = gwarp; tl < TT; tl += gwarps) {
            const int i = tl == gwarp ? i_pre : owner_of(tl, npop, tile_base);
            const FusedPop &p = PP[i];
            const uint32_t P = (uint32_t)(4 * p.N), T = S[i].T;
            const uint32_t q = (tl - p.tile_base) * 32u + lane;
            const uint32_t f = tl == gwarp ? f_pre : (q < P ? ldcg32(p.fit[src] + q) : 0u);
            if (psel) {
                // probabilistic selection: in-tile weight prefixes and the tile's weight
                const unsigned long long sum = psel_tile(f, q < P, p.cw + (size_t)(tl - p.tile_base) * 32u, lane);
                if (lane == 0)
                    p.tmask[tl - p.tile_base] = sum;
                continue;
            }
            const uint32_t lt = __ballot_sync(FULL, q < P && f < T);
            const uint32_t eq = __ballot_sync(FULL, q < P && f == T);
            if (lane == 0)
                p.tmask[tl - p.tile_base] = (unsigned long long)lt | ((unsigned long long)eq << 32);
        }
        // block-local histogram offsets of the next generation (read after
        // the barrier's bar.sync)
        if (tid == 0 && !psel) {
            uint32_t off = 0;
            for (int i = 0; i < npop; ++i) {
                const uint32_t nb = hbuckets(S[i].capn, S[i].hlon, S[i].shiftn);
                S[i].boff = off + nb <= kHistSmem ? off : 0xFFFFFFFFu;
                if (off + nb <= kHistSmem)
                    off += nb;
            }
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
                    v[r] = ldcg64(PP[i].tmask + (tt - PP[i].tile_base));
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
        if (tid == 0)
            s_next = 0u;
        __syncthreads();
        block_scan_chunks_u64(
            TT,
            [&](uint32_t e) {
                const unsigned long long v = tm[e];
                if (psel)
                    return v;  // the tile's weight
                return ((unsigned long long)__popc((uint32_t)v) << 32) | (unsigned long long)__popc((uint32_t)(v >> 32));
            },
            ex, s_tmp64);
        if (tid < npop && psel) {
            const FusedPop &p = PP[tid];
            PopSel &s = S[tid];
            const uint32_t last = p.tile_base + p.ntiles - 1u;
            s.pbase = ex[p.tile_base];
            s.pW = ex[last] + tm[last] - s.pbase;
            s.bor = 0u;
            s.bbest = ~0ull;
            if (s.pW == 0ull)
                atomicOr(err, ERR_INTERNAL);
        } else if (tid < npop) {
            const FusedPop &p = PP[tid];
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
        // m <= 32: two or four threads per pair (FusedPop::tpp)
        for (uint32_t w = gwarp; w < nwork_t; w += gwarps) {
            const uint32_t u = w * 32u;
            // the population whose (32-aligned) thread range holds this warp
            int i = -1;
            for (int j = 0; j < npop; ++j)
                if (PP[j].m <= 32 && u >= PP[j].work_base)
                    i = (i < 0 || PP[j].work_base >= PP[i].work_base) ? j : i;
            const FusedPop &p = PP[i < 0 ? 0 : i];
            const bool two = p.tpp == 2;
            const uint32_t local = u + (uint32_t)lane - p.work_base;
            const uint32_t k = two ? local >> 1 : local >> 2;
            const int half = (int)(two ? (local & 1u) : ((local >> 1) & 1u)), sub = (int)(local & 1u);
            const bool valid = i >= 0 && k < (uint32_t)p.N;
            const uint32_t gen = S[i < 0 ? 0 : i].gen0 + 1u + (uint32_t)t;
            Pre pre = pre0;
            if (w != gwarp && valid)
                pre = make_pre(p, gen, (uint32_t)t, k, half, psel);
            uint32_t fv[2] = {0u, 0u}, sl[2] = {0u, 0u};
            const PopSel &s = S[i < 0 ? 0 : i];
            switch (p.m) {
#define HADGA_PT(MM)                                                                                        \
    case MM:                                                                                                \
        if (two)                                                                                            \
            pair_thread<MM, 2>(p, s, src, gen, pre, k, half, sub, valid, sv, err, fv, sl);                  \
        else                                                                                                \
            pair_thread<MM, 4>(p, s, src, gen, pre, k, half, sub, valid, sv, err, fv, sl);                  \
        break;
                HADGA_PT(4) HADGA_PT(8) HADGA_PT(12) HADGA_PT(16) HADGA_PT(20) HADGA_PT(24) HADGA_PT(28) HADGA_PT(32)
#undef HADGA_PT
            default:
                break;
            }
            uint32_t orr = 0;
            unsigned long long key = ~0ull;
            for (int e = 0; e < (two ? 2 : 1); ++e) {
                if (psel) {
                    // no histogram: the next selection weighs every individual
                } else if (s.boff != 0xFFFFFFFFu) {
                    if (valid && fv[e] <= s.capn)
                        atomicAdd(bhist + s.boff + hkey(fv[e], s.hlon, s.shiftn), 1u);
                } else {
                    warp_hist_add(hist_of(p, par ^ 1), valid && fv[e] <= s.capn, hkey(fv[e], s.hlon, s.shiftn));
                }
                orr |= valid ? fv[e] : 0u;
                const unsigned long long ke = valid ? (((unsigned long long)fv[e] << 32) | sl[e]) : ~0ull;
                key = ke < key ? ke : key;
            }
            orr = warp_or(orr);
            key = warp_min_u64(key);
            if (lane == 0 && i >= 0) {
                atomicOr(&S[i].bor, orr);
                atomicMin(&S[i].bbest, key);
            }
        }
        // 32 < m <= 128: a warp per offspring (items 2k + half).  The block
        // owns items blockIdx.x + q * nblocks, q = 0, 1, ...; its warps take
        // the next q from a shared counter, so offspring of uneven cost (the
        // incremental path's cross block grows with c (m - c)) even out
        // within the block.
        for (;;) {
            uint32_t q = 0;
            if (lane == 0)
                q = atomicAdd(&s_next, 1u);
            q = __shfl_sync(FULL, q, 0);
            const uint32_t it = blockIdx.x + q * nblocks;
            if (it >= prm.warp_items)
                break;
            int i = -1;
            for (int j = 0; j < npop; ++j)
                if (PP[j].m > 32 && it >= PP[j].work_base &&
                    it < PP[j].work_base + 2u * (uint32_t)PP[j].N)
                    i = j;
            if (i < 0)
                continue;
            const FusedPop &p = PP[i];
            const uint32_t item = it - p.work_base, k = item >> 1;
            const int half = (int)(item & 1u);
            uint32_t *hn = hist_of(p, par ^ 1);
            const uint32_t gen = S[i].gen0 + 1u + (uint32_t)t;
            switch (p.W) {
            case 2: offspring_warp<2, INC>(p, S[i], src, gen, (uint32_t)t, k, half, sv, err, wbuf, ring, prm.inc_ring, &s_incbar[wib], inc_parity, hn, bhist); break;
            case 3: offspring_warp<3, INC>(p, S[i], src, gen, (uint32_t)t, k, half, sv, err, wbuf, ring, prm.inc_ring, &s_incbar[wib], inc_parity, hn, bhist); break;
            case 4: offspring_warp<4, INC>(p, S[i], src, gen, (uint32_t)t, k, half, sv, err, wbuf, ring, prm.inc_ring, &s_incbar[wib], inc_parity, hn, bhist); break;
            default: break;
            }
        }
        // one flush per block of its histogram counts, OR word and best key
        __syncthreads();
        for (int i = 0; i < npop; ++i) {
            const uint32_t bo = S[i].boff;
            if (bo == 0xFFFFFFFFu)
                continue;
            const uint32_t nb = hbuckets(S[i].capn, S[i].hlon, S[i].shiftn);
            uint32_t *hn = hist_of(PP[i], par ^ 1);
            for (uint32_t e = tid; e < nb; e += blockDim.x) {
                const uint32_t c = bhist[bo + e];
                if (c)
                    atomicAdd(hn + e, c);
            }
        }
        if (tid < npop) {
            const FusedPop &p = PP[tid];
            if (S[tid].bor)
                atomicOr(stat_of(p) + 1 + (par ^ 1), S[tid].bor);
            if (S[tid].bbest != ~0ull)
                atomicMin(p.traj + (S[tid].gen0 + (uint32_t)t) % (uint32_t)p.traj_cap, S[tid].bbest);
        }
        // split barrier: the next generation's first draws overlap its latency
        grid_arrive(prm.bar);
        if (t + 1 < prm.ngen)
            pre_next = first_pre(t + 1);
        if (!grid_wait(prm.bar, nblocks, epoch, err))
            return;
        src ^= 1;
        if (tid < npop) {
            S[tid].cap = S[tid].capn;
            S[tid].shift = S[tid].shiftn;
            S[tid].hlo = S[tid].hlon;
        }
        done = t + 1;
        if (prm.stop_at_zero) {
            const FusedPop &p = PP[0];
            const unsigned long long key = ldcg64(p.traj + (S[0].gen0 + (uint32_t)t) % (uint32_t)p.traj_cap);
            if ((key >> 32) == 0ull)
                break;
        }
        __syncthreads();
    }
    if (blockIdx.x == 0 && tid == 0)
        *prm.done = done;
    if (blockIdx.x == 0 && tid < npop)
        *PP[tid].gen_dev = S[tid].gen0 + (uint32_t)done;
}

size_t fused_smem_bytes(const FusedParams &p)
{
    bool inc = false;
    for (int i = 0; i < p.npop; ++i)
        inc = inc || p.p[i].gram != nullptr;
    const size_t ring_words = inc ? (size_t)(kFusedThreads / 32) * (size_t)p.inc_ring * 4u : 0u;
    const size_t r1 = std::max((size_t)4 * p.total_tiles + ring_words, (size_t)2 * kHistSmem);
    return (r1 + kHistSmem + (size_t)(kFusedThreads / 32) * p.warp_buf_words) * 4u;
}

size_t fused_smem_limit()
{
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes f0{}, f1{};
    cudaFuncGetAttributes(&f0, k_fused<false>);
    cudaFuncGetAttributes(&f1, k_fused<true>);
    const size_t stat = std::max(f0.sharedSizeBytes, f1.sharedSizeBytes);
    return (size_t)optin > stat ? (size_t)optin - stat : 0u;
}

void fused_plan_ring(FusedParams &p)
{
    // every copy of one offspring (the largest IncCopyPlan total over the
    // cuts) when the shared memory of a block allows it, else the largest
    // multiple of 32 groups that fits, at least 128
    int max_groups = 0;
    bool inc = false;
    for (int i = 0; i < p.npop; ++i)
        if (p.p[i].gram != nullptr) {
            inc = true;
            for (int c = 1; c < p.p[i].m; ++c)
                max_groups = std::max(max_groups, IncCopyPlan(p.p[i].m, c).total);
        }
    p.inc_ring = 0;
    if (!inc)
        return;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, k_fused<true>);
    const long long budget = (long long)optin - (long long)fa.sharedSizeBytes;
    int ring = (max_groups + 31) / 32 * 32;
    for (; ring > 128; ring -= 32) {
        p.inc_ring = ring;
        if ((long long)fused_smem_bytes(p) <= budget)
            return;
    }
    p.inc_ring = 128;
}

cudaError_t fused_grid(size_t smem, int *grid)
{
    cudaError_t e = cudaFuncSetAttribute(k_fused<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fused<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    int dev = 0, sms = 0, per0 = 0, per1 = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per0, k_fused<false>, kFusedThreads, smem);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per1, k_fused<true>, kFusedThreads, smem);
    if (e != cudaSuccess)
        return e;
    if (per0 < 1 || per1 < 1)
        return cudaErrorCooperativeLaunchTooLarge;
    *grid = sms;  // one resident block per SM
    return cudaSuccess;
}

cudaError_t launch_fused(const FusedParams &p, int grid, size_t smem, cudaStream_t s)
{
    bool inc = false;
    for (int i = 0; i < p.npop; ++i)
        inc = inc || p.p[i].gram != nullptr;
    void *args[] = {(void *)&p};
    const void *fn = inc ? (const void *)k_fused<true> : (const void *)k_fused<false>;
    cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kFusedThreads), args, smem, s);
    if (e == cudaSuccess)
        note_launches(1);
    return e;
}

} // namespace hadga
