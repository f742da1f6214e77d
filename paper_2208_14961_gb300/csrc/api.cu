// api.cu -- the extern "C" entry points of libhadga (declared, with the
// passages of the paper they implement, in include/hadga.h).
#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "hadga.h"
#include "common.cuh"
#include "kernels.cuh"

using namespace hadga;

namespace {

thread_local std::string g_thread_error;
std::atomic<unsigned long long> g_launches{0};
// test hook: allocations still to fail (ga_debug_fail_allocations)
std::atomic<int> g_fail_allocs{0};

// cudaMalloc, or a simulated out-of-memory while the test hook is armed
cudaError_t dev_alloc(void **p, size_t bytes)
{
    int n = g_fail_allocs.load();
    while (n > 0) {
        if (g_fail_allocs.compare_exchange_weak(n, n - 1))
            return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

constexpr int32_t kVersion = 1 * 10000 + 0 * 100 + 0;
constexpr int64_t kMaxP = int64_t(1) << 31;

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Host-side NVTX range for the duration of a scope: calls and chunks of the
// library appear by name in tools that record NVTX (ncu --nvtx, Nsight
// Systems); without such a tool attached the calls do nothing.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

} // namespace

struct ga_ctx {
    ga_config cfg;
    int m = 0, W = 0;
    int64_t N = 0, P = 0;
    size_t mat_bytes = 0;
    void *pop = nullptr;
    uint32_t *fit = nullptr;
    cudaStream_t stream = nullptr;
    int device = 0;
    uint32_t gen = 0;

    // workspace (one allocation)
    void *ws = nullptr;
    size_t ws_bytes = 0;
    void *scratch_pop = nullptr;   // P matrices: selection target, fused ping-pong
    uint32_t *scratch_fit = nullptr;
    SelWork sel{};
    unsigned long long *traj = nullptr;
    unsigned long long *best = nullptr;
    uint32_t *err = nullptr;
    // fused path
    uint32_t *bits[2] = {nullptr, nullptr};  // bit-storage ping-pong (int8 contexts)
    uint32_t *ffit = nullptr;                 // second fitness buffer
    uint32_t *fstate = nullptr;               // kFusedStateWords selection state
    uint32_t *fmisc = nullptr;                // [0] grid-barrier counter, [1] generations done, [2] generation
    int fused_blocks = 0;                     // persistent blocks (0: one per SM)
    int shape_tpp = 0;                        // m <= 32: threads per pair (0: default 4)
    int shape_nch = 0;                        // m > 32: warp Gram chunks per column (0: cost model)
    unsigned long long *ftmask = nullptr;
    uint32_t *fperm = nullptr;                // [chunk][2N] survivor orders
    unsigned long long *fperm_keys = nullptr; // [chunk][2N] sort keys when 2N > kPermSmemMax
    int fused_ok = 0;
    std::string fused_why;                    // why the persistent kernel cannot run this context
    int strict = 0;                           // ga_step: GA_EUNSUPPORTED instead of the plain path
    // incremental Gram-delta mode (BITS, 32 < m <= 128)
    int incremental = 0;
    int gram_valid = 0;
    float auto_full_ms = 0.f, auto_inc_ms = 0.f;  // ms per generation measured by the AUTO choice
    int dpad = 0;
    void *gram_mem = nullptr;                 // gram | gidx[0] | gidx[1] | counts
    int8_t *gram = nullptr;
    uint32_t *gidx[2] = {nullptr, nullptr};
    unsigned long long *gcounts = nullptr;

    // opt-in event profile of ga_step's kernels
    int profiling = 0;
    std::vector<cudaEvent_t> prof_perm, prof_fused;  // start/stop pairs

    std::string msg;
};

namespace hadga {
void note_launches(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }
void set_thread_error(const char *msg) { g_thread_error = msg; }
} // namespace hadga

namespace {

ga_status set_error(ga_ctx *c, ga_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c)
        c->msg = buf;
    else
        g_thread_error = buf;
    return st;
}

ga_status cuda_check(ga_ctx *c, cudaError_t e, const char *what)
{
    if (e == cudaSuccess)
        return GA_OK;
    if (e == cudaErrorMemoryAllocation)
        return set_error(c, GA_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    return set_error(c, GA_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

void drop_events(std::vector<cudaEvent_t> &v)
{
    for (cudaEvent_t e : v)
        cudaEventDestroy(e);
    v.clear();
}

ga_status check_storage_m(ga_ctx *c, int32_t storage, int32_t m)
{
    if (m < 4 || m > kMaxM || (m & 3))
        return set_error(c, GA_EINVAL, "order m=%d must be a multiple of 4 in [4, %d]", m, kMaxM);
    if (storage < GA_STORE_INT8 || storage > GA_STORE_BF16)
        return set_error(c, GA_EINVAL, "unknown storage %d", storage);
    return GA_OK;
}

// Constant of the fused kernel: chunk of generations whose survivor orders
// are computed together before the persistent launch.
constexpr int kChunk = 64;

// GA_PATH_AUTO by storage, order and fitness, from the measured Gram sweep
// on GB300 (8 GiB populations, m = 32..256): bit storage always takes
// popcount; int8 takes the warp-level tensor-core row Gram (FP8 operands
// from the int8 signs) for F_sq up to m = 128 and popcount otherwise; e4m3
// storage takes the tcgen05 path for F_sq at m = 128 and 256 and the
// warp-level FP8 MMA otherwise (HBM-bound at m <= 64; F1 / F2; orders the
// tcgen05 kernel does not tile); bf16 storage takes tcgen05.
// Measured overrides of GA_PATH_AUTO (ga_set_auto_path, set by the
// autotuner), by storage, order / 4 and fitness kind; 0 = none.
std::atomic<int> g_auto_override[4][kMaxM / 4 + 1][3];

int auto_path(int storage, int m, int kind)
{
    if (storage >= 0 && storage < 4 && m >= 4 && m <= kMaxM && (m & 3) == 0 && kind >= 0 && kind < 3) {
        const int o = g_auto_override[storage][m / 4][kind].load(std::memory_order_relaxed);
        if (o != 0)
            return o;
    }
    if (storage == GA_STORE_E4M3)
        return (kind == GA_FIT_SQ && (m == 128 || m == 256)) ? GA_PATH_FP8 : GA_PATH_FP8_WARP;
    if (storage == GA_STORE_BF16)
        return GA_PATH_BF16;
    if (storage == GA_STORE_INT8 && kind == GA_FIT_SQ && m % 32 == 0 && m <= 128)
        return GA_PATH_IMMA;
    return GA_PATH_POPC;
}

} // namespace

extern "C" {

int32_t ga_version(void) { return kVersion; }

ga_status ga_debug_fail_allocations(int32_t n)
{
    if (n < 0)
        return set_error(nullptr, GA_EINVAL, "n=%d must be >= 0", n);
    g_fail_allocs.store(n);
    return GA_OK;
}

uint64_t ga_kernel_launches(void) { return (uint64_t)g_launches.load(); }

size_t ga_storage_bytes(int32_t storage, int32_t m)
{
    if (m < 4 || m > kMaxM || (m & 3))
        return 0;
    return matrix_bytes(storage, m);
}

const char *ga_last_error(const ga_ctx *ctx) { return ctx ? ctx->msg.c_str() : g_thread_error.c_str(); }

ga_status ga_create(const ga_config *cfg, void *pop_dev, uint32_t *fit_dev, void *stream, ga_ctx **out)
{
    if (!out)
        return set_error(nullptr, GA_EINVAL, "out is NULL");
    *out = nullptr;
    if (!cfg)
        return set_error(nullptr, GA_EINVAL, "cfg is NULL");
    ga_status st = check_storage_m(nullptr, cfg->storage, cfg->m);
    if (st != GA_OK)
        return st;
    if (cfg->storage != GA_STORE_INT8 && cfg->storage != GA_STORE_BITS)
        return set_error(nullptr, GA_EINVAL, "a GA context stores INT8 or BITS, got %d", cfg->storage);
    if (cfg->N < 1 || 4 * cfg->N > kMaxP)
        return set_error(nullptr, GA_EINVAL, "N=%lld out of range [1, 2^29]", (long long)cfg->N);
    if (cfg->NC < 1 || cfg->NC > 64 || cfg->NR < 1 || cfg->NR > 64)
        return set_error(nullptr, GA_EINVAL, "NC=%d, NR=%d must lie in [1, 64]", cfg->NC, cfg->NR);
    if (cfg->fitness < GA_FIT_SQ || cfg->fitness > GA_FIT_NNZ)
        return set_error(nullptr, GA_EINVAL, "unknown fitness %d", cfg->fitness);
    if (cfg->traj_cap < 1)
        return set_error(nullptr, GA_EINVAL, "traj_cap must be >= 1");
    if (cfg->mutation != 0 && cfg->mutation != 1)
        return set_error(nullptr, GA_EINVAL, "mutation must be 0 (per offspring) or 1 (one draw per generation)");
    if (cfg->selection != GA_SEL_TRUNCATION && cfg->selection != GA_SEL_PROBABILISTIC)
        return set_error(nullptr, GA_EINVAL, "selection must be 0 (truncation) or 1 (probabilistic)");
    int path = cfg->path == GA_PATH_AUTO ? auto_path(cfg->storage, cfg->m, cfg->fitness) : cfg->path;
    if (!fitness_path_supported(cfg->storage, cfg->m, path))
        return set_error(nullptr, GA_EINVAL, "Gram path %d does not read storage %d", cfg->path, cfg->storage);
    if (!pop_dev || !fit_dev)
        return set_error(nullptr, GA_EINVAL, "population and fitness buffers must not be NULL");
    if (!aligned16(pop_dev) || !aligned16(fit_dev))
        return set_error(nullptr, GA_EINVAL, "population and fitness buffers must be 16-byte aligned");

    ga_ctx *c = new ga_ctx();
    c->cfg = *cfg;
    c->cfg.path = path;
    c->m = cfg->m;
    c->W = words_per_col(cfg->m);
    c->N = cfg->N;
    c->P = 4 * cfg->N;
    c->mat_bytes = matrix_bytes(cfg->storage, cfg->m);
    c->pop = pop_dev;
    c->fit = fit_dev;
    c->stream = (cudaStream_t)stream;
    cudaGetDevice(&c->device);

    const int64_t P = c->P, n_keep = 2 * c->N, tiles = (P + 31) / 32;
    const size_t bits_bytes = (size_t)P * c->m * c->W * 4u;
    // can the persistent kernel run this population alone?  (orders up to
    // kFusedMaxM, tiles up to kFusedMaxTiles, and its shared memory: the
    // tile masks and their prefix, the staged histograms, the warp buffers)
    bool fused_fit = c->m <= kFusedMaxM && (uint64_t)tiles <= kFusedMaxTiles;
    if (!fused_fit) {
        c->fused_why = c->m > kFusedMaxM ? "the persistent kernel builds orders m <= 128"
                                         : "the persistent kernel takes P <= 262144 (8192 tiles of 32 slots)";
    } else {
        FusedParams fp{};
        fp.npop = 1;
        fp.total_tiles = (uint32_t)tiles;
        fp.warp_buf_words = c->m > 32 ? ((2 * c->m * c->W + col_set_words(c->m, c->W) + 3) & ~3) : 0;
        fp.p[0].N = c->N;
        const size_t need = fused_smem_bytes(fp), have = fused_smem_limit();
        if (need > have) {
            fused_fit = false;
            char why[160];
            snprintf(why, sizeof(why), "the persistent kernel would need %zu bytes of shared memory per block (%zu "
                     "available) at m=%d, P=%lld", need, have, c->m, (long long)P);
            c->fused_why = why;
        }
    }
    // sub-allocation plan
    struct Part {
        void **dst;
        size_t bytes;
    };
    void *tmp_ptrs[32] = {};
    std::vector<Part> parts = {
        {&c->scratch_pop, (size_t)P * c->mat_bytes},
        {(void **)&c->scratch_fit, (size_t)P * 4u},
        {(void **)&c->sel.hist, 2048u * 4u},
        {(void **)&c->sel.state, sizeof(SelState)},
        {(void **)&c->sel.tmask, (size_t)tiles * 8u},
        {(void **)&c->sel.survmask, (size_t)tiles * 4u},
        {(void **)&c->sel.survbefore, (size_t)tiles * 4u},
        {(void **)&c->sel.perm, (size_t)n_keep * 4u},
        {(void **)&c->traj, (size_t)cfg->traj_cap * 8u},
        {(void **)&c->best, 8u},
        {(void **)&c->err, 4u},
    };
    if (cfg->selection == GA_SEL_PROBABILISTIC) {
        parts.push_back({(void **)&c->sel.cw, (size_t)tiles * 32u * 8u});
        parts.push_back({(void **)&c->sel.tex, (size_t)tiles * 8u});
        parts.push_back({(void **)&c->sel.wtotal, 8u});
    }
    if ((uint64_t)n_keep > kPermSmemMax) {
        const int nb = perm_global_bits((uint32_t)n_keep);
        parts.push_back({(void **)&c->sel.perm_keys, (size_t)n_keep * 8u});
        parts.push_back({(void **)&c->sel.perm_cnt, (size_t)2u * (1u << nb) * 4u});
    }
    if (fused_fit) {
        if (cfg->storage == GA_STORE_INT8) {
            parts.push_back({(void **)&c->bits[0], bits_bytes});
            parts.push_back({(void **)&c->bits[1], bits_bytes});
        }
        parts.push_back({(void **)&c->ffit, (size_t)P * 4u});
        parts.push_back({(void **)&c->fstate, kFusedStateWords * 4u});
        parts.push_back({(void **)&c->fmisc, 64u * 4u});
        parts.push_back({(void **)&c->ftmask, (size_t)tiles * 8u});
        parts.push_back({(void **)&c->fperm, (size_t)kChunk * n_keep * 4u});
        if ((uint64_t)n_keep > kPermSmemMax)
            parts.push_back({(void **)&c->fperm_keys, (size_t)kChunk * n_keep * 8u});
    }
    (void)tmp_ptrs;
    size_t total = 0;
    for (auto &p : parts)
        total = align_up(total, 256) + align_up(p.bytes, 256);
    void *ws = nullptr;
    cudaError_t e = dev_alloc(&ws, total);
    if (e != cudaSuccess) {
        delete c;
        cudaGetLastError();
        return set_error(nullptr, e == cudaErrorMemoryAllocation ? GA_ENOMEM : GA_ECUDA,
                         "workspace allocation of %zu bytes failed: %s", total, cudaGetErrorString(e));
    }
    c->ws = ws;
    c->ws_bytes = total;
    size_t off = 0;
    for (auto &p : parts) {
        off = align_up(off, 256);
        *p.dst = (char *)ws + off;
        off += align_up(p.bytes, 256);
    }
    c->sel.err = c->err;
    e = cudaMemsetAsync(ws, 0, total, c->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(c->traj, 0xFF, (size_t)cfg->traj_cap * 8u, c->stream);
    if (e != cudaSuccess) {
        cudaFree(ws);
        delete c;
        return set_error(nullptr, GA_ECUDA, "workspace initialisation failed: %s", cudaGetErrorString(e));
    }
    c->fused_ok = fused_fit ? 1 : 0;
    *out = c;
    return GA_OK;
}

ga_status ga_destroy(ga_ctx *ctx)
{
    if (!ctx)
        return GA_OK;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    drop_events(ctx->prof_perm);
    drop_events(ctx->prof_fused);
    cudaFree(ctx->gram_mem);
    cudaFree(ctx->ws);
    delete ctx;
    return GA_OK;
}

static ga_status begin(ga_ctx *ctx)
{
    if (!ctx)
        return set_error(nullptr, GA_EINVAL, "ctx is NULL");
    cudaError_t e = cudaSetDevice(ctx->device);
    return cuda_check(ctx, e, "cudaSetDevice");
}

ga_status ga_init_population(ga_ctx *ctx)
{
    NvtxRange nvtx("ga_init_population");
    ga_status st = begin(ctx);
    if (st != GA_OK)
        return st;
    st = cuda_check(ctx,
                    launch_init(ctx->pop, ctx->cfg.storage, ctx->m, 0, ctx->P, ctx->cfg.seed, ctx->cfg.pop_id,
                                ctx->stream),
                    "init");
    if (st != GA_OK)
        return st;
    ctx->gen = 0;
    ctx->gram_valid = 0;
    return cuda_check(ctx, cudaMemsetAsync(ctx->traj, 0xFF, (size_t)ctx->cfg.traj_cap * 8u, ctx->stream),
                      "trajectory reset");
}

ga_status ga_fitness(ga_ctx *ctx, int64_t first, int64_t count)
{
    NvtxRange nvtx("ga_fitness");
    ga_status st = begin(ctx);
    if (st != GA_OK)
        return st;
    if (first < 0 || count < 0 || first + count > ctx->P)
        return set_error(ctx, GA_EINVAL, "slot range [%lld, %lld) outside [0, %lld)", (long long)first,
                         (long long)(first + count), (long long)ctx->P);
    return cuda_check(ctx,
                      launch_fitness(ctx->pop, ctx->cfg.storage, ctx->m, first, count, ctx->cfg.fitness,
                                     ctx->cfg.path, ctx->fit, ctx->stream),
                      "fitness");
}

ga_status ga_select(ga_ctx *ctx)
{
    NvtxRange nvtx("ga_select");
    ga_status st = begin(ctx);
    if (st != GA_OK)
        return st;
    const uint32_t g = ctx->gen + 1u;
    ctx->gram_valid = 0;
    if (ctx->cfg.selection == GA_SEL_PROBABILISTIC)
        st = cuda_check(ctx,
                        launch_select_prob(ctx->pop, ctx->fit, ctx->N, ctx->mat_bytes, ctx->cfg.seed,
                                           ctx->cfg.pop_id, g, ctx->sel, ctx->scratch_pop, ctx->scratch_fit,
                                           ctx->stream),
                        "probabilistic select");
    else
        st = cuda_check(ctx,
                        launch_select(ctx->pop, ctx->fit, ctx->N, ctx->mat_bytes, ctx->cfg.seed, ctx->cfg.pop_id, g,
                                      ctx->sel, ctx->scratch_pop, ctx->scratch_fit, ctx->stream),
                        "select");
    if (st != GA_OK)
        return st;
    const int64_t n_keep = 2 * ctx->N;
    cudaError_t e = cudaMemcpyAsync(ctx->pop, ctx->scratch_pop, (size_t)n_keep * ctx->mat_bytes,
                                    cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->fit, ctx->scratch_fit, (size_t)n_keep * 4u, cudaMemcpyDeviceToDevice, ctx->stream);
    st = cuda_check(ctx, e, "select copy-back");
    if (st == GA_OK)
        ctx->gen = g;
    return st;
}

ga_status ga_crossover(ga_ctx *ctx)
{
    NvtxRange nvtx("ga_crossover");
    ga_status st = begin(ctx);
    if (st != GA_OK)
        return st;
    ctx->gram_valid = 0;
    return cuda_check(ctx,
                      launch_crossover(ctx->pop, ctx->cfg.storage, ctx->m, ctx->N, ctx->cfg.seed, ctx->cfg.pop_id,
                                       ctx->gen, ctx->stream),
                      "crossover");
}

ga_status ga_mutate(ga_ctx *ctx)
{
    NvtxRange nvtx("ga_mutate");
    ga_status st = begin(ctx);
    if (st != GA_OK)
        return st;
    ctx->gram_valid = 0;
    return cuda_check(ctx,
                      launch_mutate(ctx->pop, ctx->cfg.storage, ctx->m, ctx->N, ctx->cfg.NC, ctx->cfg.NR,
                                    ctx->cfg.seed, ctx->cfg.pop_id, ctx->gen, ctx->cfg.mutation, ctx->stream),
                      "mutate");
}

ga_status ga_record_best(ga_ctx *ctx)
{
    ga_status st = begin(ctx);
    if (st != GA_OK)
        return st;
    if (ctx->gen == 0)
        return set_error(ctx, GA_EINVAL, "no generation to record (generation 0)");
    unsigned long long *slot = ctx->traj + (ctx->gen - 1u) % (uint32_t)ctx->cfg.traj_cap;
    return cuda_check(ctx, launch_best(ctx->fit, ctx->P, slot, ctx->stream), "record best");
}

ga_status ga_step_plain(ga_ctx *ctx, int32_t generations)
{
    NvtxRange nvtx("ga_step_plain");
    ga_status st = begin(ctx);
    if (st != GA_OK)
        return st;
    if (generations < 0)
        return set_error(ctx, GA_EINVAL, "generations must be >= 0");
    for (int32_t t = 0; t < generations; ++t) {
        if ((st = ga_select(ctx)) != GA_OK || (st = ga_crossover(ctx)) != GA_OK || (st = ga_mutate(ctx)) != GA_OK ||
            (st = ga_fitness(ctx, 2 * ctx->N, 2 * ctx->N)) != GA_OK || (st = ga_record_best(ctx)) != GA_OK)
            return st;
    }
    return GA_OK;
}

int32_t ga_step_is_fused(const ga_ctx *ctx) { return ctx ? ctx->fused_ok : 0; }

ga_status ga_set_strict(ga_ctx *ctx, int32_t strict)
{
    if (!ctx)
        return set_error(nullptr, GA_EINVAL, "ctx is NULL");
    ctx->strict = strict ? 1 : 0;
    if (strict && !ctx->fused_ok)
        return set_error(ctx, GA_EUNSUPPORTED, "%s", ctx->fused_why.c_str());
    return GA_OK;
}

// Runs `generations` generations of ctxs[0..n) with the persistent kernel,
// in chunks of kChunk generations (survivor orders of a chunk first).
static ga_status fused_run(ga_ctx *const *ctxs, int n, int32_t generations, int stop_at_zero, int32_t *done_out,
                           bool sync_gen = true, bool tail = true)
{
    ga_ctx *c0 = ctxs[0];
    FusedParams prm{};
    memset(&prm, 0, sizeof(prm));
    prm.npop = n;
    prm.psel = c0->cfg.selection == GA_SEL_PROBABILISTIC ? 1 : 0;
    for (int i = 1; i < n; ++i)
        if (ctxs[i]->cfg.selection != c0->cfg.selection)
            return set_error(c0, GA_EUNSUPPORTED, "one persistent launch runs one selection method");
    uint32_t tiles = 0, tslots = 0, wpairs = 0;
    int max_words = 0;
    for (int i = 0; i < n; ++i) {
        ga_ctx *c = ctxs[i];
        FusedPop &p = prm.p[i];
        const bool int8 = c->cfg.storage == GA_STORE_INT8;
        p.pop[0] = int8 ? c->bits[0] : (uint32_t *)c->pop;
        p.pop[1] = int8 ? c->bits[1] : (uint32_t *)c->scratch_pop;
        p.fit[0] = c->fit;
        p.fit[1] = c->ffit;
        p.state = c->fstate;
        p.tmask = c->ftmask;
        p.cw = c->sel.cw;
        p.perm = c->fperm;
        p.traj = c->traj;
        p.gen_dev = c->fmisc + 2;
        p.m = c->m;
        p.W = c->W;
        p.nch = c->shape_nch > 0 ? c->shape_nch : warp_gram_chunks(c->m);
        p.tpp = c->shape_tpp == 2 ? 2 : 4;
        p.shared_mut = c->cfg.mutation;
        p.NC = c->cfg.NC;
        p.NR = c->cfg.NR;
        p.kind = c->cfg.fitness;
        p.traj_cap = c->cfg.traj_cap;
        p.N = c->N;
        p.seed = c->cfg.seed;
        p.pop_id = c->cfg.pop_id;
        p.tile_base = tiles;
        p.ntiles = (uint32_t)((c->P + 31) / 32);
        tiles += p.ntiles;
        if (c->m <= 32) {
            p.work_base = tslots;
            tslots += (uint32_t)(((int64_t)p.tpp * c->N + 31) / 32 * 32);
        } else {
            p.work_base = wpairs;
            wpairs += (uint32_t)(2 * c->N);  // one warp item per offspring
            // 16-byte aligned per warp (cp.async and vector copies of the parents)
            max_words = std::max(max_words, (2 * c->m * c->W + col_set_words(c->m, c->W) + 3) & ~3);
        }
        if (int8) {
            cudaError_t e = launch_convert(c->pop, GA_STORE_INT8, c->bits[0], GA_STORE_BITS, c->m, c->P, c0->stream);
            if (e != cudaSuccess)
                return cuda_check(c0, e, "convert to bit storage");
        }
        p.gram = nullptr;
        if (c->incremental) {
            if (!c->gram_valid) {
                cudaError_t e = launch_gram_store((const uint32_t *)c->pop, c->m, c->P, c->gram, c->dpad, c->gidx[0],
                                                  c0->stream);
                if (e != cudaSuccess)
                    return cuda_check(c0, e, "Gram store");
                c->gram_valid = 1;
            }
            p.gram = c->gram;
            p.gidx[0] = c->gidx[0];
            p.gidx[1] = c->gidx[1];
            p.dpad = c->dpad;
        }
        if (sync_gen) {
            cudaError_t e = launch_set_u32(c->fmisc + 2, c->gen, c0->stream);
            if (e != cudaSuccess)
                return cuda_check(c0, e, "generation counter");
        }
    }
    if (tiles > kFusedMaxTiles)
        return set_error(c0, GA_EUNSUPPORTED, "populations too large for one persistent launch");
    prm.total_tiles = tiles;
    prm.thread_slots = tslots;
    prm.warp_items = wpairs;
    prm.warp_buf_words = max_words;
    prm.stop_at_zero = stop_at_zero;
    prm.bar = c0->fmisc;
    prm.done = (int32_t *)(c0->fmisc + 1);
    prm.err = c0->err;
    fused_plan_ring(prm);
    const size_t smem = fused_smem_bytes(prm);
    if (smem > fused_smem_limit())
        return set_error(c0, GA_EUNSUPPORTED,
                         "the persistent kernel would need %zu bytes of shared memory per block for these "
                         "populations (%zu available)", smem, fused_smem_limit());
    int grid = 0;
    cudaError_t e = fused_grid(smem, &grid);
    if (e != cudaSuccess)
        return cuda_check(c0, e, "fused kernel occupancy");
    if (c0->fused_blocks > 0 && c0->fused_blocks < grid)
        grid = c0->fused_blocks;

    int cur = 0;
    int32_t total_done = 0;
    for (int32_t left = generations; left > 0;) {
        const int chunk = left < kChunk ? left : kChunk;
        NvtxRange nvtx_chunk("persistent chunk");
        for (int i = 0; i < n; ++i) {
            ga_ctx *c = ctxs[i];
            cudaEvent_t ev[2] = {nullptr, nullptr};
            if (c->profiling) {
                cudaEventCreate(&ev[0]);
                cudaEventCreate(&ev[1]);
                cudaEventRecord(ev[0], c0->stream);
            }
            // the survivor orders of truncation selection (probabilistic selection draws per parent slot)
            e = prm.psel ? cudaSuccess
                         : launch_perm_table((uint32_t)(2 * c->N), c->cfg.seed, c->cfg.pop_id, c->gen + 1u, chunk,
                                             c->fperm, c0->stream, c->fmisc + 2, c->fperm_keys);
            if (c->profiling) {
                cudaEventRecord(ev[1], c0->stream);
                c->prof_perm.push_back(ev[0]);
                c->prof_perm.push_back(ev[1]);
            }
            if (e == cudaSuccess)
                e = cudaMemsetAsync(c->fstate, 0, kFusedStateWords * 4u, c0->stream);
            if (e != cudaSuccess)
                return cuda_check(c0, e, "survivor orders");
        }
        e = cudaMemsetAsync(c0->fmisc, 0, 2 * sizeof(uint32_t), c0->stream);
        if (e != cudaSuccess)
            return cuda_check(c0, e, "barrier reset");
        prm.ngen = chunk;
        prm.src = cur;
        cudaEvent_t ev[2] = {nullptr, nullptr};
        if (c0->profiling) {
            cudaEventCreate(&ev[0]);
            cudaEventCreate(&ev[1]);
            cudaEventRecord(ev[0], c0->stream);
        }
        e = launch_fused(prm, grid, smem, c0->stream);
        if (c0->profiling) {
            cudaEventRecord(ev[1], c0->stream);
            c0->prof_fused.push_back(ev[0]);
            c0->prof_fused.push_back(ev[1]);
        }
        if (e != cudaSuccess)
            return cuda_check(c0, e, "persistent generation kernel");
        int32_t ran = chunk;
        if (stop_at_zero) {
            e = cudaMemcpyAsync(&ran, c0->fmisc + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, c0->stream);
            if (e == cudaSuccess)
                e = cudaStreamSynchronize(c0->stream);
            if (e != cudaSuccess)
                return cuda_check(c0, e, "generations done");
            uint32_t err = 0;
            cudaMemcpy(&err, c0->err, 4, cudaMemcpyDeviceToHost);
            if (err)
                return ga_sync(c0);
        }
        for (int i = 0; i < n; ++i)
            ctxs[i]->gen += (uint32_t)ran;
        total_done += ran;
        cur ^= (ran & 1);
        left -= chunk;
        if (ran < chunk)
            break;
    }
    for (int i = 0; i < n && tail; ++i) {
        ga_ctx *c = ctxs[i];
        const bool int8 = c->cfg.storage == GA_STORE_INT8;
        if (int8) {
            e = launch_convert(c->bits[cur], GA_STORE_BITS, c->pop, GA_STORE_INT8, c->m, c->P, c0->stream);
        } else if (cur == 1) {
            e = cudaMemcpyAsync(c->pop, c->scratch_pop, (size_t)c->P * c->mat_bytes, cudaMemcpyDeviceToDevice,
                                c0->stream);
        }
        if (e == cudaSuccess && cur == 1)
            e = cudaMemcpyAsync(c->fit, c->ffit, (size_t)c->P * 4u, cudaMemcpyDeviceToDevice, c0->stream);
        if (e == cudaSuccess && cur == 1 && c->incremental)
            e = cudaMemcpyAsync(c->gidx[0], c->gidx[1], (size_t)c->P * 4u, cudaMemcpyDeviceToDevice, c0->stream);
        if (e != cudaSuccess)
            return cuda_check(c0, e, "copy-back of the final population");
    }
    if (done_out)
        *done_out = total_done;
    return GA_OK;
}

ga_status ga_step(ga_ctx *ctx, int32_t generations, int32_t stop_at_zero, int32_t *done)
{
    NvtxRange nvtx("ga_step");
    ga_status st = begin(ctx);
    if (st != GA_OK)
        return st;
    if (generations < 0)
        return set_error(ctx, GA_EINVAL, "generations must be >= 0");
    if (!ctx->fused_ok && ctx->strict)
        return set_error(ctx, GA_EUNSUPPORTED, "strict mode: %s", ctx->fused_why.c_str());
    if (ctx->fused_ok) {
        int32_t d = 0;
        st = fused_run(&ctx, 1, generations, stop_at_zero, &d);
        if (st == GA_OK && done) {
            if ((st = ga_sync(ctx)) != GA_OK)
                return st;
            *done = d;
        }
        return st;
    }
    int32_t n = 0;
    for (; n < generations;) {
        if ((st = ga_step_plain(ctx, 1)) != GA_OK)
            return st;
        ++n;
        if (stop_at_zero) {
            int64_t s;
            uint32_t f;
            if ((st = ga_best(ctx, &s, &f)) != GA_OK)
                return st;
            if (f == 0)
                break;
        }
    }
    if (done)
        *done = n;
    return GA_OK;
}

ga_status ga_step_multi(ga_ctx *const *ctxs, int32_t n, int32_t generations)
{
    NvtxRange nvtx("ga_step_multi");
    if (!ctxs || n < 1)
        return set_error(nullptr, GA_EINVAL, "ctxs must hold n >= 1 contexts");
    if (generations < 0)
        return set_error(nullptr, GA_EINVAL, "generations must be >= 0");
    bool fused = n <= kMaxPops, strict = false;
    for (int32_t i = 0; i < n; ++i) {
        if (!ctxs[i])
            return set_error(nullptr, GA_EINVAL, "context %d is NULL", i);
        if (ctxs[i]->stream != ctxs[0]->stream || ctxs[i]->device != ctxs[0]->device)
            return set_error(nullptr, GA_EINVAL, "contexts must share stream and device");
        fused = fused && ctxs[i]->fused_ok && ctxs[i]->cfg.selection == ctxs[0]->cfg.selection;
        strict = strict || ctxs[i]->strict;
    }
    if (!fused && strict)
        return set_error(nullptr, GA_EUNSUPPORTED, "strict mode: the populations cannot run in one persistent launch "
                         "(more than %d, or one of them cannot run the persistent kernel)", kMaxPops);
    ga_status st = begin(ctxs[0]);
    if (st != GA_OK)
        return st;
    if (fused) {
        st = fused_run(ctxs, n, generations, 0, nullptr);
        if (st != GA_OK)
            return set_error(nullptr, st, "%s", ga_last_error(ctxs[0]));
        return GA_OK;
    }
    for (int32_t i = 0; i < n; ++i) {
        st = ga_step_plain(ctxs[i], generations);
        if (st != GA_OK)
            return set_error(nullptr, st, "population %d: %s", i, ga_last_error(ctxs[i]));
    }
    return GA_OK;
}

ga_status ga_profile(ga_ctx *ctx, int32_t enable)
{
    ga_status st = begin(ctx);
    if (st != GA_OK)
        return st;
    cudaStreamSynchronize(ctx->stream);
    drop_events(ctx->prof_perm);
    drop_events(ctx->prof_fused);
    ctx->profiling = enable ? 1 : 0;
    return GA_OK;
}

static float sum_pairs(const std::vector<cudaEvent_t> &v)
{
    float total = 0.f;
    for (size_t i = 0; i + 1 < v.size(); i += 2) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, v[i], v[i + 1]) == cudaSuccess)
            total += ms;
    }
    return total;
}

ga_status ga_profile_read(ga_ctx *ctx, float *perm_ms, float *fused_ms, int32_t *fused_launches)
{
    ga_status st = begin(ctx);
    if (st != GA_OK)
        return st;
    if (!perm_ms || !fused_ms || !fused_launches)
        return set_error(ctx, GA_EINVAL, "NULL output");
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess)
        return cuda_check(ctx, e, "profile sync");
    *perm_ms = sum_pairs(ctx->prof_perm);
    *fused_ms = sum_pairs(ctx->prof_fused);
    *fused_launches = (int32_t)(ctx->prof_fused.size() / 2);
    return GA_OK;
}

ga_status ga_step_multi_graph(ga_ctx *const *ctxs, int32_t n, int32_t generations, int32_t chunk)
{
    NvtxRange nvtx("ga_step_multi_graph");
    if (!ctxs || n < 1 || n > kMaxPops)
        return set_error(nullptr, GA_EINVAL, "ctxs must hold 1..%d contexts", kMaxPops);
    if (generations < 0 || chunk < 2 || chunk > kChunk || (chunk & 1))
        return set_error(nullptr, GA_EINVAL, "chunk must be even and in [2, %d]", kChunk);
    for (int32_t i = 0; i < n; ++i) {
        if (!ctxs[i])
            return set_error(nullptr, GA_EINVAL, "context %d is NULL", i);
        if (ctxs[i]->stream != ctxs[0]->stream || ctxs[i]->device != ctxs[0]->device)
            return set_error(nullptr, GA_EINVAL, "contexts must share stream and device");
        if (!ctxs[i]->fused_ok || ctxs[i]->cfg.storage != GA_STORE_BITS)
            return set_error(nullptr, GA_EUNSUPPORTED, "graph replay needs fused-capable BITS contexts");
        if (!ctxs[i]->stream)
            return set_error(nullptr, GA_EINVAL, "graph capture needs a non-default stream");
    }
    ga_status st = begin(ctxs[0]);
    if (st != GA_OK)
        return st;
    ga_ctx *c0 = ctxs[0];
    const int32_t reps = generations / chunk, rem = generations % chunk;
    if (reps > 0) {
        // stale incremental Gram storage is rebuilt outside the captured chunk
        for (int32_t i = 0; i < n; ++i) {
            ga_ctx *c = ctxs[i];
            if (c->incremental && !c->gram_valid) {
                cudaError_t e = launch_gram_store((const uint32_t *)c->pop, c->m, c->P, c->gram, c->dpad, c->gidx[0],
                                                  c0->stream);
                if (e != cudaSuccess)
                    return set_error(nullptr, GA_ECUDA, "Gram store: %s", cudaGetErrorString(e));
                c->gram_valid = 1;
            }
        }
        // device generation counters take over from here
        for (int32_t i = 0; i < n; ++i) {
            cudaError_t e = launch_set_u32(ctxs[i]->fmisc + 2, ctxs[i]->gen, c0->stream);
            if (e != cudaSuccess)
                return set_error(nullptr, GA_ECUDA, "generation counter: %s", cudaGetErrorString(e));
        }
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        cudaError_t e = cudaStreamBeginCapture(c0->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess)
            return set_error(nullptr, GA_ECUDA, "begin capture: %s", cudaGetErrorString(e));
        // one chunk, even length: the ping-pong buffers end where they started
        st = fused_run(ctxs, n, chunk, 0, nullptr, false, false);
        e = cudaStreamEndCapture(c0->stream, &graph);
        if (st != GA_OK || e != cudaSuccess) {
            if (graph)
                cudaGraphDestroy(graph);
            cudaGetLastError();
            return set_error(nullptr, st != GA_OK ? st : GA_ECUDA, "capture of a chunk failed: %s",
                             st != GA_OK ? ga_last_error(c0) : cudaGetErrorString(e));
        }
        // the capture advanced the host counters without running; undo that
        for (int32_t i = 0; i < n; ++i)
            ctxs[i]->gen -= (uint32_t)chunk;
        e = cudaGraphInstantiate(&exec, graph, 0);
        if (e == cudaSuccess) {
            for (int32_t r = 0; r < reps && e == cudaSuccess; ++r)
                e = cudaGraphLaunch(exec, c0->stream);
            cudaGraphExecDestroy(exec);
        }
        cudaGraphDestroy(graph);
        if (e != cudaSuccess)
            return set_error(nullptr, GA_ECUDA, "graph replay: %s", cudaGetErrorString(e));
        // the capture counted one chunk's kernels once; every replay runs them
        note_launches((reps - 1) * (n + 1));
        for (int32_t i = 0; i < n; ++i)
            ctxs[i]->gen += (uint32_t)(reps * chunk);
    }
    if (rem > 0)
        return ga_step_multi(ctxs, n, rem);
    return GA_OK;
}

static ga_status incremental_auto(ga_ctx *ctx);

ga_status ga_set_incremental(ga_ctx *ctx, int32_t enable)
{
    ga_status st = begin(ctx);
    if (st != GA_OK)
        return st;
    if (enable < 0 || enable > 2)
        return set_error(ctx, GA_EINVAL, "enable must be 0 (off), 1 (on) or 2 (choose by measurement)");
    if (enable == 2)
        return incremental_auto(ctx);
    if (!enable) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(ctx->gram_mem);
        ctx->gram_mem = nullptr;
        ctx->gram = nullptr;
        ctx->gidx[0] = ctx->gidx[1] = nullptr;
        ctx->gcounts = nullptr;
        ctx->incremental = 0;
        ctx->gram_valid = 0;
        return GA_OK;
    }
    if (ctx->cfg.storage != GA_STORE_BITS || ctx->m <= 32 || ctx->m > 128 || !ctx->fused_ok)
        return set_error(ctx, GA_EUNSUPPORTED,
                         "incremental Gram mode needs BITS storage, 32 < m <= 128 and a fused-capable context");
    if (ctx->cfg.selection != GA_SEL_TRUNCATION)
        return set_error(ctx, GA_EUNSUPPORTED,
                         "incremental Gram mode needs truncation selection (parents and offspring trade Gram "
                         "buffers one to one; probabilistic selection may draw an individual twice)");
    if (!ctx->gram_mem) {
        const int dpad = gram_tiles(ctx->m) * 64;  // 8 x 8 int8 tiles of the upper triangle
        const size_t gbytes = align_up((size_t)ctx->P * dpad, 256), ibytes = align_up((size_t)ctx->P * 4u, 256);
        void *mem = nullptr;
        cudaError_t e = dev_alloc(&mem, gbytes + 2 * ibytes + 256);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_error(ctx, e == cudaErrorMemoryAllocation ? GA_ENOMEM : GA_ECUDA,
                             "Gram storage of %zu bytes: %s", gbytes + 2 * ibytes + 256, cudaGetErrorString(e));
        }
        ctx->gram_mem = mem;
        ctx->dpad = dpad;
        ctx->gram = (int8_t *)mem;
        ctx->gidx[0] = (uint32_t *)((char *)mem + gbytes);
        ctx->gidx[1] = (uint32_t *)((char *)mem + gbytes + ibytes);
        ctx->gcounts = (unsigned long long *)((char *)mem + gbytes + 2 * ibytes);
    }
    ctx->incremental = 1;
    st = cuda_check(ctx,
                    launch_gram_store((const uint32_t *)ctx->pop, ctx->m, ctx->P, ctx->gram, ctx->dpad, ctx->gidx[0],
                                      ctx->stream),
                    "Gram store");
    ctx->gram_valid = st == GA_OK;
    return st;
}

// GA_INC_AUTO: from the current population, time kAutoGens generations of
// the fused path with full fitness recomputation and with the stored Gram
// (after kAutoWarm untimed generations each, the same for both), restore the
// population, fitness, generation and trajectory, and keep the faster mode.
static ga_status incremental_auto(ga_ctx *ctx)
{
    constexpr int kAutoWarm = 4, kAutoGens = 32;
    // the same preconditions as enabling (reports GA_EUNSUPPORTED)
    ga_status st = ga_set_incremental(ctx, 1);
    if (st != GA_OK)
        return st;
    const size_t pop_bytes = (size_t)ctx->P * ctx->mat_bytes, fit_bytes = (size_t)ctx->P * 4u,
                 traj_bytes = (size_t)ctx->cfg.traj_cap * 8u;
    void *save = nullptr;
    cudaError_t e = dev_alloc(&save, pop_bytes + fit_bytes + traj_bytes + 64);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(ctx, e == cudaErrorMemoryAllocation ? GA_ENOMEM : GA_ECUDA,
                         "incremental AUTO: state copy: %s", cudaGetErrorString(e));
    }
    char *sp = (char *)save, *sf = sp + pop_bytes, *st_traj = sf + fit_bytes;
    const uint32_t g0 = ctx->gen;
    auto copy = [&](void *dst, const void *src, size_t n) {
        return cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToDevice, ctx->stream);
    };
    e = copy(sp, ctx->pop, pop_bytes);
    if (e == cudaSuccess)
        e = copy(sf, ctx->fit, fit_bytes);
    if (e == cudaSuccess)
        e = copy(st_traj, ctx->traj, traj_bytes);
    auto restore = [&]() {
        cudaError_t r = copy(ctx->pop, sp, pop_bytes);
        if (r == cudaSuccess)
            r = copy(ctx->fit, sf, fit_bytes);
        if (r == cudaSuccess)
            r = copy(ctx->traj, st_traj, traj_bytes);
        ctx->gen = g0;
        ctx->gram_valid = 0;
        return r;
    };
    float ms[2] = {0.f, 0.f};
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (e == cudaSuccess)
        e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess)
        e = cudaEventCreate(&ev[1]);
    for (int mode = 0; mode < 2 && e == cudaSuccess && st == GA_OK; ++mode) {
        ctx->incremental = mode;
        if (mode == 1) {
            e = launch_gram_store((const uint32_t *)ctx->pop, ctx->m, ctx->P, ctx->gram, ctx->dpad, ctx->gidx[0],
                                  ctx->stream);
            ctx->gram_valid = e == cudaSuccess;
        }
        if (e == cudaSuccess)
            st = fused_run(&ctx, 1, kAutoWarm, 0, nullptr);
        if (st == GA_OK && e == cudaSuccess)
            e = cudaEventRecord(ev[0], ctx->stream);
        if (st == GA_OK && e == cudaSuccess)
            st = fused_run(&ctx, 1, kAutoGens, 0, nullptr);
        if (st == GA_OK && e == cudaSuccess)
            e = cudaEventRecord(ev[1], ctx->stream);
        if (st == GA_OK && e == cudaSuccess)
            e = cudaEventSynchronize(ev[1]);
        if (st == GA_OK && e == cudaSuccess)
            e = cudaEventElapsedTime(&ms[mode], ev[0], ev[1]);
        if (st == GA_OK && e == cudaSuccess)
            st = ga_sync(ctx);
        const cudaError_t r = restore();
        if (e == cudaSuccess)
            e = r;
    }
    for (cudaEvent_t x : ev)
        if (x)
            cudaEventDestroy(x);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(ctx->stream);
    cudaFree(save);
    if (st != GA_OK)
        return st;
    if (e != cudaSuccess)
        return cuda_check(ctx, e, "incremental AUTO");
    ctx->auto_full_ms = ms[0] / kAutoGens;
    ctx->auto_inc_ms = ms[1] / kAutoGens;
    if (ms[1] < ms[0]) {
        ctx->incremental = 1;  // the Gram of the restored population is rebuilt by the next ga_step
        return GA_OK;
    }
    ctx->incremental = 1;
    return ga_set_incremental(ctx, 0);
}

ga_status ga_get_incremental(const ga_ctx *ctx, int32_t *enabled, float *full_ms_per_gen, float *inc_ms_per_gen)
{
    if (!ctx || !enabled || !full_ms_per_gen || !inc_ms_per_gen)
        return set_error(nullptr, GA_EINVAL, "NULL argument");
    *enabled = ctx->incremental;
    *full_ms_per_gen = ctx->auto_full_ms;
    *inc_ms_per_gen = ctx->auto_inc_ms;
    return GA_OK;
}

ga_status ga_check_incremental(ga_ctx *ctx, uint64_t *entry_mismatch, uint64_t *fit_mismatch)
{
    ga_status st = begin(ctx);
    if (st != GA_OK)
        return st;
    if (!entry_mismatch || !fit_mismatch)
        return set_error(ctx, GA_EINVAL, "NULL output");
    if (!ctx->incremental)
        return set_error(ctx, GA_EINVAL, "incremental mode is off");
    if (!ctx->gram_valid)
        return set_error(ctx, GA_EINVAL, "the Gram storage is stale (population changed outside ga_step)");
    cudaError_t e = cudaMemsetAsync(ctx->gcounts, 0, 16, ctx->stream);
    if (e == cudaSuccess)
        e = launch_gram_check((const uint32_t *)ctx->pop, ctx->m, ctx->P, ctx->cfg.fitness, ctx->gram, ctx->dpad,
                              ctx->gidx[0], ctx->fit, ctx->gcounts, ctx->stream);
    unsigned long long h[2] = {0, 0};
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h, ctx->gcounts, 16, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess)
        return cuda_check(ctx, e, "incremental check");
    *entry_mismatch = h[0];
    *fit_mismatch = h[1];
    return GA_OK;
}

ga_status ga_get_gram(ga_ctx *ctx, int64_t slot, int32_t *host_G)
{
    ga_status st = begin(ctx);
    if (st != GA_OK)
        return st;
    if (!host_G || slot < 0 || slot >= ctx->P)
        return set_error(ctx, GA_EINVAL, "bad slot %lld or NULL output", (long long)slot);
    if (!ctx->incremental || !ctx->gram_valid)
        return set_error(ctx, GA_EINVAL, "no current incremental Gram storage");
    uint32_t g = 0;
    cudaError_t e = cudaMemcpyAsync(&g, ctx->gidx[0] + slot, 4, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess)
        return cuda_check(ctx, e, "Gram index read");
    if ((int64_t)g >= ctx->P)
        return set_error(ctx, GA_ECUDA, "Gram index %u of slot %lld out of range", g, (long long)slot);
    const int m = ctx->m, nb = gram_tiles_nb(m);
    std::vector<int8_t> h((size_t)ctx->dpad);
    e = cudaMemcpy(h.data(), ctx->gram + (size_t)g * ctx->dpad, (size_t)ctx->dpad, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return cuda_check(ctx, e, "Gram read");
    for (int i = 0; i < m; ++i) {
        host_G[i * m + i] = m;
        for (int j = i + 1; j < m; ++j) {
            const int I = i >> 3, J = j >> 3, t = I * nb - I * (I - 1) / 2 + (J - I);
            host_G[i * m + j] = host_G[j * m + i] = 2 * (int32_t)h[(size_t)t * 64 + (i & 7) * 8 + (j & 7)];
        }
    }
    return GA_OK;
}

ga_status ga_set_fused_shape(ga_ctx *ctx, int32_t tpp, int32_t nch)
{
    if (!ctx)
        return set_error(nullptr, GA_EINVAL, "ctx is NULL");
    if (tpp != 0 && tpp != 2 && tpp != 4)
        return set_error(ctx, GA_EINVAL, "threads per pair must be 0 (default), 2 or 4");
    if (nch < 0 || nch > 16 || (nch > 0 && nch > ctx->m / 2))
        return set_error(ctx, GA_EINVAL, "nch=%d must be 0 (cost model) or in [1, min(16, m/2)]", nch);
    ctx->shape_tpp = tpp;
    ctx->shape_nch = nch;
    return GA_OK;
}

ga_status ga_set_auto_path(int32_t storage, int32_t m, int32_t kind, int32_t path)
{
    ga_status st = check_storage_m(nullptr, storage, m);
    if (st != GA_OK)
        return st;
    if (kind < GA_FIT_SQ || kind > GA_FIT_NNZ)
        return set_error(nullptr, GA_EINVAL, "unknown fitness %d", kind);
    if (path < GA_PATH_AUTO || path > GA_PATH_FP8_WARP)
        return set_error(nullptr, GA_EINVAL, "unknown path %d", path);
    if (path != GA_PATH_AUTO) {
        const bool tc = path == GA_PATH_FP8 || path == GA_PATH_BF16;
        const bool ok = tc ? ((path == GA_PATH_FP8) == (storage == GA_STORE_E4M3) &&
                              (path == GA_PATH_BF16) == (storage == GA_STORE_BF16) && kind == GA_FIT_SQ &&
                              fitness_tc_supported(storage, m))
                           : fitness_path_supported(storage, m, path);
        if (!ok)
            return set_error(nullptr, GA_EINVAL, "path %d cannot compute fitness %d of storage %d at m=%d", path, kind,
                             storage, m);
    }
    g_auto_override[storage][m / 4][kind].store(path, std::memory_order_relaxed);
    return GA_OK;
}

ga_status ga_set_fused_grid(ga_ctx *ctx, int32_t blocks)
{
    if (!ctx || blocks < 0)
        return set_error(nullptr, GA_EINVAL, "bad context or block count");
    ctx->fused_blocks = blocks;
    return GA_OK;
}

ga_status ga_sync(ga_ctx *ctx)
{
    ga_status st = begin(ctx);
    if (st != GA_OK)
        return st;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess)
        return cuda_check(ctx, e, "stream synchronize");
    uint32_t err = 0;
    e = cudaMemcpy(&err, ctx->err, 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return cuda_check(ctx, e, "error word read");
    if (err & ERR_TIMEOUT)
        return set_error(ctx, GA_ETIMEOUT, "a grid barrier wait exceeded its budget (device error word 0x%x)", err);
    if (err)
        return set_error(ctx, GA_ECUDA, "device-side check failed (device error word 0x%x)", err);
    return GA_OK;
}

ga_status ga_best(ga_ctx *ctx, int64_t *slot, uint32_t *fitness)
{
    ga_status st = begin(ctx);
    if (st != GA_OK)
        return st;
    if (!slot || !fitness)
        return set_error(ctx, GA_EINVAL, "slot and fitness must not be NULL");
    st = cuda_check(ctx, launch_best(ctx->fit, ctx->P, ctx->best, ctx->stream), "best");
    if (st != GA_OK)
        return st;
    unsigned long long key = 0;
    cudaError_t e = cudaMemcpyAsync(&key, ctx->best, 8, cudaMemcpyDeviceToHost, ctx->stream);
    if (e != cudaSuccess)
        return cuda_check(ctx, e, "best read");
    if ((st = ga_sync(ctx)) != GA_OK)
        return st;
    *fitness = (uint32_t)(key >> 32);
    *slot = (int64_t)(uint32_t)key;
    return GA_OK;
}

ga_status ga_trajectory(ga_ctx *ctx, uint32_t *host_fit, int64_t *host_slot, int32_t cap, int32_t *n)
{
    ga_status st = begin(ctx);
    if (st != GA_OK)
        return st;
    if (!host_fit || !host_slot || !n || cap < 0)
        return set_error(ctx, GA_EINVAL, "bad trajectory arguments");
    const int32_t tc = ctx->cfg.traj_cap;
    std::vector<unsigned long long> keys((size_t)tc);
    cudaError_t e = cudaMemcpyAsync(keys.data(), ctx->traj, (size_t)tc * 8u, cudaMemcpyDeviceToHost, ctx->stream);
    if (e != cudaSuccess)
        return cuda_check(ctx, e, "trajectory read");
    if ((st = ga_sync(ctx)) != GA_OK)
        return st;
    const uint32_t g = ctx->gen;
    int32_t have = (int32_t)(g < (uint32_t)tc ? g : (uint32_t)tc);
    if (have > cap)
        have = cap;
    const uint32_t g_first = g - (uint32_t)have + 1u;
    for (int32_t i = 0; i < have; ++i) {
        const unsigned long long k = keys[(g_first + (uint32_t)i - 1u) % (uint32_t)tc];
        host_fit[i] = (uint32_t)(k >> 32);
        host_slot[i] = (int64_t)(uint32_t)k;
    }
    *n = have;
    return GA_OK;
}

ga_status ga_generation(const ga_ctx *ctx, uint32_t *g)
{
    if (!ctx || !g)
        return set_error(nullptr, GA_EINVAL, "ctx and g must not be NULL");
    *g = ctx->gen;
    return GA_OK;
}

ga_status ga_set_generation(ga_ctx *ctx, uint32_t g)
{
    if (!ctx)
        return set_error(nullptr, GA_EINVAL, "ctx is NULL");
    ctx->gen = g;
    return GA_OK;
}

ga_status ga_set_slot(ga_ctx *ctx, int64_t slot, const int8_t *host_matrix)
{
    ga_status st = begin(ctx);
    if (st != GA_OK)
        return st;
    if (!host_matrix || slot < 0 || slot >= ctx->P)
        return set_error(ctx, GA_EINVAL, "bad slot %lld or NULL matrix", (long long)slot);
    const int m = ctx->m;
    ctx->gram_valid = 0;
    for (int i = 0; i < m * m; ++i)
        if (host_matrix[i] != 1 && host_matrix[i] != -1)
            return set_error(ctx, GA_EINVAL, "entry %d of the matrix is %d, not +1 or -1", i, host_matrix[i]);
    std::vector<uint8_t> buf(ctx->mat_bytes);
    if (ctx->cfg.storage == GA_STORE_INT8) {
        memcpy(buf.data(), host_matrix, ctx->mat_bytes);
    } else {
        std::vector<uint32_t> w((size_t)m * ctx->W, 0u);
        for (int j = 0; j < m; ++j)
            for (int i = 0; i < m; ++i)
                if (host_matrix[i * m + j] < 0)
                    w[(size_t)j * ctx->W + (i >> 5)] |= 1u << (i & 31);
        memcpy(buf.data(), w.data(), ctx->mat_bytes);
    }
    cudaError_t e = cudaMemcpyAsync((char *)ctx->pop + (size_t)slot * ctx->mat_bytes, buf.data(), ctx->mat_bytes,
                                    cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(ctx->stream);
    return cuda_check(ctx, e, "set slot");
}

ga_status ga_get_slot(ga_ctx *ctx, int64_t slot, int8_t *host_matrix)
{
    ga_status st = begin(ctx);
    if (st != GA_OK)
        return st;
    if (!host_matrix || slot < 0 || slot >= ctx->P)
        return set_error(ctx, GA_EINVAL, "bad slot %lld or NULL matrix", (long long)slot);
    std::vector<uint8_t> buf(ctx->mat_bytes);
    cudaError_t e = cudaMemcpyAsync(buf.data(), (const char *)ctx->pop + (size_t)slot * ctx->mat_bytes,
                                    ctx->mat_bytes, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(ctx->stream);
    if ((st = cuda_check(ctx, e, "get slot")) != GA_OK)
        return st;
    const int m = ctx->m;
    if (ctx->cfg.storage == GA_STORE_INT8) {
        memcpy(host_matrix, buf.data(), ctx->mat_bytes);
    } else {
        const uint32_t *w = (const uint32_t *)buf.data();
        for (int j = 0; j < m; ++j)
            for (int i = 0; i < m; ++i)
                host_matrix[i * m + j] = ((w[(size_t)j * ctx->W + (i >> 5)] >> (i & 31)) & 1u) ? -1 : 1;
    }
    return GA_OK;
}

ga_status ga_init_batch(void *pop_dev, int32_t storage, int32_t m, int64_t P, uint32_t seed, uint32_t pop_id,
                        void *stream)
{
    ga_status st = check_storage_m(nullptr, storage, m);
    if (st != GA_OK)
        return st;
    if (!pop_dev || !aligned16(pop_dev) || P < 0 || P > kMaxP)
        return set_error(nullptr, GA_EINVAL, "bad population buffer or P");
    return cuda_check(nullptr, launch_init(pop_dev, storage, m, 0, P, seed, pop_id, (cudaStream_t)stream), "init");
}

ga_status ga_fitness_batch(const void *pop_dev, int32_t storage, int32_t m, int64_t P, int32_t kind, int32_t path,
                           uint32_t *fit_dev, void *stream)
{
    ga_status st = check_storage_m(nullptr, storage, m);
    if (st != GA_OK)
        return st;
    if (!pop_dev || !fit_dev || !aligned16(pop_dev) || !aligned16(fit_dev) || P < 0 || P > kMaxP)
        return set_error(nullptr, GA_EINVAL, "bad buffers or P");
    if (kind < GA_FIT_SQ || kind > GA_FIT_NNZ)
        return set_error(nullptr, GA_EINVAL, "unknown fitness %d", kind);
    if (path == GA_PATH_AUTO)
        path = auto_path(storage, m, kind);
    cudaStream_t s = (cudaStream_t)stream;
    if (path == GA_PATH_FP8 || path == GA_PATH_BF16) {
        if ((path == GA_PATH_FP8) != (storage == GA_STORE_E4M3) || (path == GA_PATH_BF16) != (storage == GA_STORE_BF16))
            return set_error(nullptr, GA_EINVAL, "path %d does not read storage %d", path, storage);
        if (!fitness_tc_supported(storage, m))
            return set_error(nullptr, GA_EUNSUPPORTED, "tensor-core path not available for m=%d", m);
        if (kind != GA_FIT_SQ)
            return set_error(nullptr, GA_EUNSUPPORTED, "tensor-core paths compute the sum-of-squares fitness only");
        return cuda_check(nullptr, launch_fitness_tc(pop_dev, storage, m, 0, P, kind, fit_dev, nullptr, s),
                          "tensor-core fitness");
    }
    if (path < GA_PATH_AUTO || path > GA_PATH_FP8_WARP || !fitness_path_supported(storage, m, path))
        return set_error(nullptr, GA_EINVAL, "path %d does not read storage %d", path, storage);
    return cuda_check(nullptr, launch_fitness(pop_dev, storage, m, 0, P, kind, path, fit_dev, s), "fitness");
}

ga_status ga_gram_real_batch(const void *q_dev, void *g_dev, int32_t type, int32_t m, int64_t B, void *stream)
{
    if (type != GA_REAL_F32 && type != GA_REAL_F64)
        return set_error(nullptr, GA_EINVAL, "unknown real type %d", type);
    if (m < 1 || m > 256)
        return set_error(nullptr, GA_EINVAL, "m=%d outside 1..256", m);
    if (B == 0)
        return GA_OK;  // nothing to do; empty buffers may be NULL
    if (!q_dev || !g_dev || !aligned16(q_dev) || !aligned16(g_dev) || B < 0 || B > kMaxP)
        return set_error(nullptr, GA_EINVAL, "bad buffers or B");
    const size_t bytes = (size_t)B * m * m * (type == GA_REAL_F64 ? 8u : 4u);
    const uintptr_t q0 = (uintptr_t)q_dev, g0 = (uintptr_t)g_dev;
    if (B > 0 && q0 < g0 + bytes && g0 < q0 + bytes)
        return set_error(nullptr, GA_EINVAL, "q and g overlap");
    return cuda_check(nullptr, launch_gram_real(q_dev, g_dev, type == GA_REAL_F64, m, B, (cudaStream_t)stream),
                      "real Gram");
}

ga_status ga_convert(const void *src, int32_t src_storage, void *dst, int32_t dst_storage, int32_t m, int64_t P,
                     void *stream)
{
    ga_status st = check_storage_m(nullptr, src_storage, m);
    if (st != GA_OK)
        return st;
    if ((st = check_storage_m(nullptr, dst_storage, m)) != GA_OK)
        return st;
    if (!src || !dst || !aligned16(src) || !aligned16(dst) || P < 0 || P > kMaxP)
        return set_error(nullptr, GA_EINVAL, "bad buffers or P");
    return cuda_check(nullptr, launch_convert(src, src_storage, dst, dst_storage, m, P, (cudaStream_t)stream),
                      "convert");
}

} // extern "C"
