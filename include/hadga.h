/*
 * hadga.h -- C ABI of libhadga, the GB300 (sm_103a) implementation of the
 * per-generation population step of the genetic algorithm for Hadamard
 * matrices of Balogh & Ruiz (arXiv 2208.14961).
 *
 * The library computes everything on the GPU.  Callers own the population
 * and fitness buffers (device memory, e.g. torch tensors) and the CUDA
 * stream; a context borrows them and owns only its workspace.
 *
 * Conventions shared by every entry point
 *  - Status: every call returns a ga_status and never aborts the process.
 *    The text of the last failure of a context is ga_last_error(ctx); calls
 *    without a context report through ga_last_error(NULL) (per thread).
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy
 *    default stream).  Every call is stream-ordered and returns without
 *    waiting for the GPU, except where marked "synchronises".
 *  - Device errors (a grid-barrier wait that ran out, an internal check)
 *    raise bits in a device error word; synchronising calls turn them into
 *    GA_ETIMEOUT or GA_ECUDA.
 *
 * Population (Sec. 3.1, Eq. (1)-(2)): P = 4N matrices of order m = 4k,
 * slots [0, 2N) parents P_1..P_2N, slots [2N, 4N) offspring O_1..O_2N.
 * Storage formats of one matrix Q (rows i, columns j, entries +1 / -1):
 *  - GA_STORE_INT8 : m*m int8, row-major, Q[i][j] at byte i*m + j (the
 *                    paper's layout, Sec. 3.4); values 1 and -1.
 *  - GA_STORE_BITS : m*W uint32 words, W = ceil(m/32); column j occupies
 *                    words [j*W, j*W + W); bit r of word w is 1 iff
 *                    Q[32w + r][j] == -1; bits of rows >= m are 0.
 *  - GA_STORE_E4M3 : m*m bytes row-major, FP8 e4m3: +1 = 0x38, -1 = 0xB8.
 *  - GA_STORE_BF16 : m*m uint16 row-major, bfloat16: +1 = 0x3F80, -1 = 0xBF80.
 * Buffers must be 16-byte aligned.  Fitness values are uint32 (all three
 * fitness functions are below 2^32 for m <= 256).
 *
 * Randomness: Philox4x32-10 (Salmon et al., SC'11), key (seed, pop_id),
 * counter (op, generation, index, (sub << 16) | block); op INIT = 0,
 * SELECT = 1, CROSS = 2, MUTATE = 3, CONFIG = 4 (mixed-order sizes),
 * PSELECT = 5 (probabilistic selection: words 0, 1 of (PSELECT, g, p, 0)
 * form the 64-bit draw of parent slot p).  A word w gives an integer in
 * [lo, hi] as lo + floor(w * (hi - lo + 1) / 2^32).
 *
 * Tracing: every host call, and each chunk of the persistent kernel, is an
 * NVTX range named after the call ("ga_step", "persistent chunk", ...).
 */
#ifndef HADGA_H
#define HADGA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GA_OK = 0,
    GA_EINVAL = 1,        /* bad argument (null pointer, misaligned, out of range) */
    GA_ENOMEM = 2,        /* workspace allocation failed */
    GA_ECUDA = 3,         /* a CUDA call or kernel failed */
    GA_ETIMEOUT = 4,      /* a bounded device wait gave up */
    GA_EUNSUPPORTED = 5   /* valid request this build does not provide */
} ga_status;

/* Fitness of a matrix from its column Gram G = Q^T Q (Sec. 3.2). */
typedef enum {
    GA_FIT_SQ = 0,  /* sum over i < j of G_ij^2 */
    GA_FIT_ABS = 1, /* F1 = sum_{i,j} |G_ij| - m^2          (Eq. (3), (8)) */
    GA_FIT_NNZ = 2  /* F2 = number of nonzero G_ij - m      (Eq. (4), (9)) */
} ga_fitness_kind;

typedef enum {
    GA_STORE_INT8 = 0,
    GA_STORE_BITS = 1,
    GA_STORE_E4M3 = 2,
    GA_STORE_BF16 = 3
} ga_storage;

/* How the Gram contraction of ga_fitness / ga_fitness_batch is computed.
 * Every path is exact; they differ only in speed and accepted storage. */
typedef enum {
    GA_PATH_AUTO = 0,   /* fastest measured exact path for storage, m and fitness */
    GA_PATH_INT32 = 1,  /* int8 storage, CUDA-core 8-bit dot products */
    GA_PATH_IMMA = 2,   /* int8 storage, warp-level tensor-core MMA (mma.sync with FP8
                           operands converted from the int8 signs, FP32 accumulate) */
    GA_PATH_FP8 = 3,    /* e4m3 storage, tcgen05 tensor cores, FP32 accumulate */
    GA_PATH_BF16 = 4,   /* bf16 storage, tcgen05 tensor cores, FP32 accumulate */
    GA_PATH_POPC = 5,   /* bits (or int8) storage, XOR + population count */
    GA_PATH_FP8_WARP = 6 /* e4m3 storage, warp-level FP8 tensor-core MMA (mma.sync), FP32 accumulate */
} ga_gram_path;

typedef struct {
    int32_t m;        /* order, multiple of 4, 4 <= m <= 256 */
    int32_t NC;       /* columns mutated per offspring, 1 <= NC <= 64 (Sec. 3.5) */
    int64_t N;        /* P = 4N, N >= 1 */
    uint32_t seed;    /* Philox key word 0 */
    uint32_t pop_id;  /* Philox key word 1 */
    int32_t NR;       /* row pairs per mutated column, 1 <= NR <= 64 */
    int32_t fitness;  /* ga_fitness_kind */
    int32_t storage;  /* GA_STORE_INT8 or GA_STORE_BITS */
    int32_t path;     /* ga_gram_path used by ga_fitness */
    int32_t traj_cap; /* generations kept in the best-fitness trajectory (>= 1) */
    int32_t mutation; /* 0: each offspring draws its own columns and rows (methods 2 and 3
                         of Sec. 3.5); 1: method 1 of Sec. 3.5, every offspring of a
                         generation uses the same draws, those of stream index 2N */
    int32_t selection; /* ga_selection: 0 truncation (Sec. 3.3, the paper's method);
                          1 probabilistic, probabilities inverse to the fitness (the
                          variant Sec. 3.3 names): weights floor(2^32 / (F + 1)), each
                          parent slot p drawn independently with replacement by
                          t = floor(u W / 2^64), u the 64 bits of Philox
                          (PSELECT = 5, g, p, 0) words 0 and 1, W the sum of the
                          weights; the parent is the individual whose cumulative-weight
                          interval holds t.  Not with the incremental mode. */
} ga_config;

typedef enum { GA_SEL_TRUNCATION = 0, GA_SEL_PROBABILISTIC = 1 } ga_selection;

typedef struct ga_ctx ga_ctx;

/* Library version (major * 10000 + minor * 100 + patch). */
int32_t ga_version(void);

/* Bytes of one matrix of order m in `storage` (0 for invalid arguments). */
size_t ga_storage_bytes(int32_t storage, int32_t m);

/* Creates a context over caller-owned buffers.
 *   pop_dev : device buffer of 4N matrices in cfg->storage (INT8 or BITS).
 *   fit_dev : device uint32 [4N], fitness of every slot.
 *   stream  : cudaStream_t for every call on the context.
 * Allocates the workspace (about one extra population plus O(N) words) on
 * the current device.  The buffers must outlive the context.  The
 * generation counter starts at 0.  Errors: GA_EINVAL, GA_ENOMEM, GA_ECUDA. */
ga_status ga_create(const ga_config *cfg, void *pop_dev, uint32_t *fit_dev, void *stream, ga_ctx **out);

/* Frees the workspace (synchronises the stream).  NULL is accepted. */
ga_status ga_destroy(ga_ctx *ctx);

/* a1 -- initial population (Sec. 3.1; Sec. 6, population set-up and the
 * column-shuffle kernel).  Column 0 of every slot is all +1; column j >= 1
 * starts as (m/2) x (-1) over (m/2) x (+1) and is shuffled by Fisher-Yates,
 * swapping entry i1 with i1 + U[0, m-1-i1] for i1 = 0..m-2, with the words
 * of stream (INIT, 0, slot, j).  Resets the generation counter and the
 * trajectory.  Does not compute fitness (call ga_fitness). */
ga_status ga_init_population(ga_ctx *ctx);

/* a2 -- fitness of slots [first, first + count) (Sec. 3.2, Eq. (3)-(5)),
 * by the context's Gram path.  Exact integers.  GA_EINVAL if the range
 * leaves [0, 4N). */
ga_status ga_fitness(ga_ctx *ctx, int64_t first, int64_t count);

/* a3 + a4 -- truncation selection with random placement (Sec. 3.3; Sec. 6,
 * the selection line).  Starts generation g + 1.  The 2N slots that come
 * first in ascending (F, slot) order survive; listed in increasing slot
 * order s_0 < ... < s_{2N-1}, parent slot p receives matrix and fitness of
 * s_{pi(p)}, where pi sorts the keys (u_d, d), u_d = word (d mod 4) of
 * Philox block (SELECT, g + 1, floor(d/4), 0).  Offspring slots keep their
 * old contents until ga_crossover. */
ga_status ga_select(ga_ctx *ctx);

/* a5 -- column-exchange crossover of generation g (Sec. 3.4, Fig. 2,
 * Eq. (6)).  Pair k in [0, N) with cut c = U[1, m-1] from stream
 * (CROSS, g, k, 0): slot 2N+k = P_k[:, :c] | P_{N+k}[:, c:] and
 * slot 3N+k = P_{N+k}[:, :c] | P_k[:, c:]. */
ga_status ga_crossover(ga_ctx *ctx);

/* a6 -- balanced pair-flip mutation, method 3 (Sec. 3.5, Eq. (7), Fig. 3),
 * generation g.  Offspring o in [0, 2N) (slot 2N+o) draws NC columns in
 * [1, m-1], then NR first rows and NR second rows in [0, m-1], from stream
 * (MUTATE, g, o, 0); for each column in order and each pair in order, the
 * two entries are negated iff their signs differ.  With cfg.mutation = 1
 * (method 1) every offspring uses the draws of stream (MUTATE, g, 2N, 0). */
ga_status ga_mutate(ga_ctx *ctx);

/* a8 -- records the best (least F, lowest slot) of the current population
 * as the trajectory entry of the current generation. */
ga_status ga_record_best(ga_ctx *ctx);

/* a1..a8 -- runs `generations` generations with one kernel per operator:
 * select, crossover, mutate, fitness of the 2N offspring, record best. */
ga_status ga_step_plain(ga_ctx *ctx, int32_t generations);

/* a1..a8 -- runs `generations` generations with the fused persistent
 * generation kernel (one cooperative launch per chunk of generations; the
 * data-independent survivor orders of a chunk are computed first).  Results
 * are bit-identical to ga_step_plain.  When stop_at_zero is set, stops after
 * the first generation whose best fitness is 0.  *done (may be NULL)
 * receives the number of generations run; it synchronises only when
 * stop_at_zero is set or done is not NULL.  The fused kernel takes orders
 * m <= 128 and P <= 262,144 whose shared-memory plan fits a block; for any
 * other population ga_step runs the plain sequence instead (see
 * ga_step_is_fused), or returns GA_EUNSUPPORTED with the reason in
 * ga_last_error when the context is strict (ga_set_strict). */
ga_status ga_step(ga_ctx *ctx, int32_t generations, int32_t stop_at_zero, int32_t *done);

/* Like ga_step for n contexts at once (orders m may differ): every
 * generation of every population runs in the same persistent launch.  All
 * contexts must share the stream and device and use BITS or INT8 storage. */
ga_status ga_step_multi(ga_ctx *const *ctxs, int32_t n, int32_t generations);

/* Like ga_step_multi, with the generations run as replays of one captured
 * CUDA graph of `chunk` generations (even, 2..64): the survivor orders, the
 * state resets and the persistent launch of a chunk are captured once and
 * replayed generations / chunk times; generation numbers are read from
 * device-side counters, so every replay continues where the last one
 * stopped.  A remainder runs through ga_step_multi.  Needs BITS contexts
 * on one non-default stream; results equal ga_step_multi. */
ga_status ga_step_multi_graph(ga_ctx *const *ctxs, int32_t n, int32_t generations, int32_t chunk);

/* a7 -- incremental Gram-delta fitness.  The paper recomputes G = Q^T Q in
 * full; this mode derives the same G from the operators' structure (the
 * fitness of Sec. 3.2 under the crossover of Sec. 3.4 and the mutation of
 * Sec. 3.5): a pair flip in column c changes only row and column c of G, by
 * -2s(Q[r1][j] - Q[r2][j]) with s = Q[r1][c]; a column exchange at cut c
 * keeps the blocks of G inside each parent's part.
 * When enabled, the context keeps every individual's Gram (G / 2 as int8
 * in 8 x 8 tiles of the upper triangle: 64 * t bytes, t = n(n+1)/2 tiles,
 * n = ceil(m/8), in a separate device allocation of P times that) and the
 * fused kernel builds each offspring's Gram from its parents' tiles: only
 * the c(m - c) cross entries, the entries of tiles cut by c and the row and
 * column of each flipped column (O(m) entries per flip) are recomputed.  Results stay bit-identical to the full
 * recomputation.  Needs BITS storage and 32 < m <= 128 on a fused-capable
 * context (GA_EUNSUPPORTED otherwise).  Enabling (re)builds the Gram of the
 * current population; ga_init_population, ga_set_slot and the one-kernel-
 * per-operator calls mark it stale and the next ga_step rebuilds it.  After
 * writing the population buffer directly, enable again.  enable = 0 frees
 * the Gram storage.  enable = 2 (AUTO) chooses by measurement: from the
 * current population it runs 4 + 32 generations of the fused path with full
 * recomputation and the same with the stored Gram, timing the last 32 of
 * each with CUDA events, restores the population, fitness, generation and
 * trajectory, and keeps the faster mode (the times are reported by
 * ga_get_incremental).  Synchronises; allocates a copy of the state for the
 * duration of the call. */
ga_status ga_set_incremental(ga_ctx *ctx, int32_t enable);

/* Whether incremental mode (the Gram-delta update of the fitness of Sec. 3.2
 * under the operators of Sec. 3.4-3.5) is on, and the milliseconds per generation the
 * last AUTO choice measured with full recomputation and with the stored
 * Gram (0 if AUTO never ran).  Host only. */
ga_status ga_get_incremental(const ga_ctx *ctx, int32_t *enabled, float *full_ms_per_gen, float *inc_ms_per_gen);

/* Full recomputation check of the incremental state: recomputes every
 * slot's Gram and fitness from the population and counts the stored
 * 4-entry Gram words (*entry_mismatch) and fitness words (*fit_mismatch)
 * that differ.  Synchronises.  GA_EINVAL unless incremental mode is on. */
ga_status ga_check_incremental(ga_ctx *ctx, uint64_t *entry_mismatch, uint64_t *fit_mismatch);

/* Stored Gram of one slot in incremental mode, expanded to the full m x m
 * int32 matrix G (diagonal m, symmetric) in host memory.  Synchronises. */
ga_status ga_get_gram(ga_ctx *ctx, int64_t slot, int32_t *host_G);

/* Number of persistent blocks of the fused kernel for launches led by ctx
 * (0 = one per SM, the default).  Chosen by the autotuner. */
ga_status ga_set_fused_grid(ga_ctx *ctx, int32_t blocks);

/* Launch shape of this population in the persistent kernel (an
 * implementation parameter with no counterpart in the paper, chosen by the
 * autotuner per order; results are identical for every shape).  tpp:
 * threads per pair of the m <= 32 build, 2 (each thread computes a whole
 * offspring) or 4 (each half of its terms); 0 = default 4.  nch: chunks per
 * column of the warp-level Gram of m > 32 (the m * nch work units of a
 * warp; 1 <= nch <= min(16, m/2)); 0 = the built-in cost model.  Host only;
 * applies from the next ga_step. */
ga_status ga_set_fused_shape(ga_ctx *ctx, int32_t tpp, int32_t nch);

/* Process-wide override of GA_PATH_AUTO for (storage, m, kind): the Gram
 * path (of the fitness of Sec. 3.2, Eq. (3)-(5)) the autotuner measured
 * fastest on this GPU (GA_PATH_AUTO clears the
 * override and restores the built-in choice).  GA_EINVAL when the path
 * cannot compute that fitness of that storage at that order.  Host only. */
ga_status ga_set_auto_path(int32_t storage, int32_t m, int32_t kind, int32_t path);

/* 1 if ga_step runs the fused kernel for this context, 0 if it falls back. */
int32_t ga_step_is_fused(const ga_ctx *ctx);

/* Execution policy (no counterpart in the paper).
 * strict != 0: ga_step and ga_step_multi never fall back to the one-kernel-
 * per-operator path; a population the persistent kernel cannot run makes
 * them return GA_EUNSUPPORTED (reason in ga_last_error).  Returns
 * GA_EUNSUPPORTED at once when setting strict mode on such a context (the
 * mode is still set), GA_OK otherwise.  Host only. */
ga_status ga_set_strict(ga_ctx *ctx, int32_t strict);

/* Best individual of the current population: least F, lowest slot on ties
 * (Sec. 6, the minimum of F).  Synchronises. */
ga_status ga_best(ga_ctx *ctx, int64_t *slot, uint32_t *fitness);

/* Copies the recorded trajectory (best fitness and slot after generations
 * max(1, g - cap + 1) .. g) to host arrays of length cap; *n receives the
 * count.  Synchronises. */
ga_status ga_trajectory(ga_ctx *ctx, uint32_t *host_fit, int64_t *host_slot, int32_t cap, int32_t *n);

/* Current generation number g (0 after ga_init_population). */
ga_status ga_generation(const ga_ctx *ctx, uint32_t *g);

/* Sets the generation counter (resuming from a saved population). */
ga_status ga_set_generation(ga_ctx *ctx, uint32_t g);

/* Waits for the stream and reports device error bits.  Synchronises. */
ga_status ga_sync(ga_ctx *ctx);

/* Copies one slot to / from a host int8 m x m row-major matrix.
 * Synchronises. */
ga_status ga_set_slot(ga_ctx *ctx, int64_t slot, const int8_t *host_matrix);
ga_status ga_get_slot(ga_ctx *ctx, int64_t slot, int8_t *host_matrix);

/* Message of the last failure of ctx (or of the calling thread when ctx is
 * NULL); never NULL. */
const char *ga_last_error(const ga_ctx *ctx);

/* ---- Test-only exports: failure detection without a fault ---------------- */

/* Drives one of the library's bounded device waits to its limit, on purpose
 * and without any fault (not a step of the paper; it checks the failure
 * handling of every kernel that waits).  which = 0: the grid-wide barrier of
 * the persistent generation kernel, launched cooperatively on two blocks
 * that expect one more arrival than there are blocks; which = 1: the
 * mbarrier wait of the tensor-core and bulk-copy pipelines, on a barrier
 * nobody arrives on.  The wait gives up after budget_us microseconds
 * (1 .. 1,000,000), records ERR_TIMEOUT (bit 0) in a fresh device error
 * word and the kernel returns normally.  Synchronises the stream, stores
 * the error word in *err_out and returns GA_ETIMEOUT when the timeout bit is
 * set (GA_OK if the wait completed, which it cannot).  The CUDA context stays
 * usable afterwards.  Allocates and frees 8 bytes of device memory. */
ga_status ga_debug_wait_timeout(int32_t which, uint32_t budget_us, uint32_t *err_out, void *stream);

/* Makes the next n device allocations of this library (context workspaces
 * of ga_create, the Gram storage of ga_set_incremental) fail as if the
 * device were out of memory, without calling the allocator: the failing call
 * returns GA_ENOMEM and leaves nothing behind (no context, no allocation).
 * n = 0 clears the hook; n < 0 is GA_EINVAL.  Process-wide. */
ga_status ga_debug_fail_allocations(int32_t n);

/* ---- Instrumentation ------------------------------------------------------ */

/* Number of kernels this library has launched in the process so far (all
 * contexts and batch calls; memsets and copies are not counted). */
uint64_t ga_kernel_launches(void);

/* When enabled, ga_step records CUDA events around its two kernels (the
 * survivor-order table and the persistent generation kernel) on the
 * context's stream; ga_profile_read returns their summed device times in
 * milliseconds since the last enable, and the number of persistent
 * launches.  Synchronises. */
ga_status ga_profile(ga_ctx *ctx, int32_t enable);
ga_status ga_profile_read(ga_ctx *ctx, float *perm_ms, float *fused_ms, int32_t *fused_launches);

/* ---- Stateless batch calls (no context) -------------------------------- */

/* a1 on a bare buffer of P matrices (the init of ga_init_population). */
ga_status ga_init_batch(void *pop_dev, int32_t storage, int32_t m, int64_t P, uint32_t seed,
                        uint32_t pop_id, void *stream);

/* a2 on a bare buffer: fitness `kind` of P matrices into fit_dev[P] using
 * `path` (GA_PATH_AUTO picks by storage).  GA_EINVAL when path and storage
 * do not match; GA_EUNSUPPORTED when the path is unavailable for m. */
ga_status ga_fitness_batch(const void *pop_dev, int32_t storage, int32_t m, int64_t P, int32_t kind,
                           int32_t path, uint32_t *fit_dev, void *stream);

/* Allocation-free selection, for callers that cannot call cudaMalloc while
 * this step runs (a framework hook that forbids device allocation, a fixed
 * workspace, a path where an allocation would synchronise the device).
 * The paper has no counterpart: this is the a3 + a4 step of ga_select
 * (generation `gen`, same survivors, same order) with its scratch in one
 * fixed device array of the library (88.5 KiB, held by every GPU that
 * loads the library until the process exits) instead of a context.
 *   pop_in, fit_in   : the population (4N matrices in `storage`, INT8 or
 *                      BITS) and its fitness, read only.
 *   parents_out,     : the 2N parents in placement order (2N matrices and
 *   parent_fit_out     2N fitness words).  Neither output may overlap
 *                      pop_in, fit_in or the other output (GA_EINVAL).
 * N is limited to 1..8192 (P <= 32768); larger N is rejected with
 * GA_EINVAL.  No cudaMalloc, cudaFree or allocating routine is called.  The
 * first call on a device looks up the array's device address (with that
 * device current); under lazy module loading (CUDA's default) it is also
 * the call that loads the library's device code on that device, which can
 * take device memory.  So make one warm-up call per device before any
 * region that forbids allocation or stream capture.  The address is kept
 * per device ordinal and is invalid once that device's context is
 * destroyed (cudaDeviceReset): do not call this entry point afterwards.
 * Every call shares the one array and leaves its contents behind (the parts
 * that must start at zero are cleared by each call), so calls that overlap
 * on the GPU -- on different streams, or from different threads -- race.
 * Stream-ordered; argument errors are reported through ga_last_error(NULL);
 * the device-side consistency checks (survivor counts and masks) raise bits
 * in the array's error word, which this call clears first and does not read:
 * ga_select_static_error reads it. */
ga_status ga_select_static(const void *pop_in, const uint32_t *fit_in, void *parents_out, uint32_t *parent_fit_out,
                           int32_t storage, int32_t m, int64_t N, uint32_t seed, uint32_t pop_id, uint32_t gen,
                           void *stream);

/* The error word of the last ga_select_static call on the current device
 * whose work is ordered before `stream`: copied into *err_out (host memory)
 * after `stream` has been synchronised.  0 when every consistency check
 * held; bit 1 (value 2) when the survivor counts or masks disagreed (a
 * parent was then clamped to the last slot and the outputs are wrong).
 * A diagnostic for tests and debugging: it synchronises, and its pageable
 * copy may take host staging memory.  GA_EINVAL for a NULL err_out,
 * GA_ECUDA for a CUDA error (message in ga_last_error(NULL)). */
ga_status ga_select_static_error(uint32_t *err_out, void *stream);

/* Element type of ga_gram_real_batch. */
typedef enum {
    GA_REAL_F32 = 0,  /* float  */
    GA_REAL_F64 = 1   /* double */
} ga_real_type;

/* The batched matrix product of the speed comparison of Sec. 2 (Table 1:
 * N = 10,000 random 100 x 100 float64 matrices, each multiplied by its own
 * transpose).  Not a step of the GA.  Computes G_b = Q_b^T Q_b for b < B:
 *   q_dev : B real m x m matrices of `type`, row-major, entry (r, i) of
 *           matrix b at q_dev[(b*m + r)*m + i]; read only.
 *   g_dev : B matrices of the same type and layout, written in full (both
 *           triangles of the symmetric G_b).
 * Entry (i, j) is the sum over r = 0 .. m-1, ascending, of Q_ri Q_rj with one
 * fused multiply-add per term in the type's precision, so it lies within
 * m u / (1 - m u) * sum_r |Q_ri Q_rj| of the exact value (u = 2^-53 for
 * double, 2^-24 for float).  1 <= m <= 256, 0 <= B <= 2^31 (B = 0 does
 * nothing and accepts NULL buffers).  Both pointers are device memory owned
 * by the caller, 16-byte aligned, and must not overlap.  GA_EINVAL for a bad type, size, pointer or
 * overlap (message in ga_last_error(NULL)).  Stream-ordered, asynchronous. */
ga_status ga_gram_real_batch(const void *q_dev, void *g_dev, int32_t type, int32_t m, int64_t B, void *stream);

/* Converts P matrices between storage formats (any pair). */
ga_status ga_convert(const void *src, int32_t src_storage, void *dst, int32_t dst_storage, int32_t m,
                     int64_t P, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* HADGA_H */
