// kernels.cuh -- host-side launch wrappers of the libhadga kernels and the
// small structs shared between the C-ABI layer and the kernel files.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace hadga {

// Bytes of one matrix of order m in a storage format.
inline size_t matrix_bytes(int storage, int m)
{
    switch (storage) {
    case 0: return (size_t)m * m;                           // int8
    case 1: return (size_t)m * ((m + 31) / 32) * 4u;        // bits
    case 2: return (size_t)m * m;                           // e4m3
    case 3: return (size_t)m * m * 2u;                      // bf16
    default: return 0;
    }
}

// Radix-select state of one selection (device memory).
struct SelState {
    uint32_t prefix;   // high bits of the threshold found so far
    uint32_t need;     // survivors still to take at the current level
    uint32_t T;        // threshold fitness: every F < T survives
    uint32_t take_eq;  // how many F == T survive (lowest slots first)
};

// Largest survivor count whose order is sorted entirely in shared memory.
constexpr uint32_t kPermSmemMax = 24576;
// Buckets of the shared-memory survivor-order sort.
constexpr int kPermSmemBits = 11;

// Adds n to the process-wide count of launched kernels (ga_kernel_launches).
void note_launches(int n);
// Sets the calling thread's message returned by ga_last_error(NULL).
void set_thread_error(const char *msg);

// ---- init (k_init.cu) -----------------------------------------------------
cudaError_t launch_init(void *pop, int storage, int m, int64_t first, int64_t count, uint32_t seed, uint32_t pop_id,
                        cudaStream_t s);

// ---- fitness (k_fitness.cu) -----------------------------------------------
// path: 1 INT32, 2 IMMA, 5 POPC (0 = AUTO resolved by the caller).
cudaError_t launch_fitness(const void *pop, int storage, int m, int64_t first, int64_t count, int kind, int path,
                           uint32_t *fit, cudaStream_t s);
bool fitness_path_supported(int storage, int m, int path);

// ---- tensor-core fitness (k_tc.cu) -----------------------------------------
cudaError_t launch_fitness_tc(const void *pop, int storage, int m, int64_t first, int64_t count, int kind,
                              uint32_t *fit, uint32_t *err, cudaStream_t s);
bool fitness_tc_supported(int storage, int m);

// ---- operators (k_ops.cu) ---------------------------------------------------
cudaError_t launch_crossover(void *pop, int storage, int m, int64_t N, uint32_t seed, uint32_t pop_id, uint32_t gen,
                             cudaStream_t s);
// shared = 1: method 1 of Sec. 3.5 (all offspring use the draws of stream index 2N).
cudaError_t launch_mutate(void *pop, int storage, int m, int64_t N, int NC, int NR, uint32_t seed, uint32_t pop_id,
                          uint32_t gen, int shared, cudaStream_t s);
// Least (F << 32 | slot) of fit[0, P) into *out (which is first set to ~0).
cudaError_t launch_best(const uint32_t *fit, int64_t P, unsigned long long *out, cudaStream_t s);
cudaError_t launch_convert(const void *src, int src_storage, void *dst, int dst_storage, int m, int64_t P,
                           cudaStream_t s);
// Batched real Gram G_b = Q_b^T Q_b (FP64 when f64 != 0, else FP32).
cudaError_t launch_gram_real(const void *q, void *g, int f64, int m, int64_t B, cudaStream_t s);
void gram_real_shape(int m, int elem, int &threads, int &kc, size_t &smem);
// Tiled half-Gram (common.cuh: 8 x 8 int8 tiles of the upper triangle of
// G / 2) of P bit-storage matrices into gram[q * dpad]; gidx[q] = q.
cudaError_t launch_gram_store(const uint32_t *pop, int m, int64_t P, int8_t *gram, int dpad, uint32_t *gidx,
                              cudaStream_t s);
// Recomputes the Gram / 2 and fitness of P bit-storage matrices and counts,
// into counts[0] / counts[1], stored entries gram[gidx[q]] and fitness words
// fit[q] that differ.
cudaError_t launch_gram_check(const uint32_t *pop, int m, int64_t P, int kind, const int8_t *gram, int dpad,
                              const uint32_t *gidx, const uint32_t *fit, unsigned long long *counts, cudaStream_t s);

// ---- selection (k_select.cu) -------------------------------------------------
struct SelWork {
    uint32_t *hist;           // 2048 counters
    SelState *state;
    unsigned long long *tmask;  // [tiles] lt | eq << 32
    uint32_t *survmask;       // [tiles]
    uint32_t *survbefore;     // [tiles]
    uint32_t *perm;           // [2N]
    unsigned long long *perm_keys;  // [2N] when 2N > kPermSmemMax
    uint32_t *perm_cnt;       // [2 * buckets] when 2N > kPermSmemMax
    uint32_t *err;
    // probabilistic selection: in-tile inclusive weight prefixes [tiles][32],
    // exclusive prefix of the tile sums [tiles], total weight [1] (the tile
    // sums themselves go to tmask)
    unsigned long long *cw, *tex, *wtotal;
};
// Selection of generation `gen`: leaves in scratch_pop[0, 2N) / scratch_fit the
// parents in placement order (matrix bytes per slot = mat_bytes).
cudaError_t launch_select(const void *pop, const uint32_t *fit, int64_t N, size_t mat_bytes, uint32_t seed,
                          uint32_t pop_id, uint32_t gen, const SelWork &w, void *scratch_pop, uint32_t *scratch_fit,
                          cudaStream_t s);
// Probabilistic selection of generation `gen` (weights inverse to F): the 2N
// drawn parents into scratch_pop[0, 2N) / scratch_fit.  Needs w.cw, w.tex,
// w.wtotal and w.tmask.
cudaError_t launch_select_prob(const void *pop, const uint32_t *fit, int64_t N, size_t mat_bytes, uint32_t seed,
                               uint32_t pop_id, uint32_t gen, const SelWork &w, void *scratch_pop,
                               uint32_t *scratch_fit, cudaStream_t s);
// Survivor orders pi of `ngen` consecutive generations into out[ngen][n],
// one block per generation.  The first generation is gen0, or *gen_dev + 1
// when gen_dev is not null (a device-side counter, so that a captured launch
// sequence can be replayed).  n <= kPermSmemMax sorts in shared memory; a
// larger n needs `keys`, ngen * n 64-bit words of device memory.
cudaError_t launch_perm_table(uint32_t n, uint32_t seed, uint32_t pop_id, uint32_t gen0, int ngen, uint32_t *out,
                              cudaStream_t s, const uint32_t *gen_dev = nullptr,
                              unsigned long long *keys = nullptr);
// *p = v, as a one-thread kernel (stream-ordered, capturable).
cudaError_t launch_set_u32(uint32_t *p, uint32_t v, cudaStream_t s);
int perm_global_bits(uint32_t n);

// ---- fused persistent generation kernel (k_fused.cu) -------------------------
constexpr int kMaxPops = 16;       // populations in one persistent launch
constexpr int kHistR = 4096;       // buckets of a selection histogram
constexpr int kFusedThreads = 512;
constexpr uint32_t kHistSmem = 8192;  // histogram words staged in shared memory per pass
constexpr int kFusedMaxM = 128;    // orders the fused kernel builds (larger: plain path)
constexpr uint32_t kFusedMaxTiles = 8192;   // joint tiles of 32 slots (P <= 262144)

// Per-population state words of the fused kernel (device memory):
// hist[2][kHistR] selection histograms by generation parity, ref[3][kHistR]
// refinement histograms, stat[4] = {max F, OR of F (parity 0, parity 1), spare}.
constexpr size_t kFusedStateWords = 5 * kHistR + 4;

struct FusedPop {
    uint32_t *pop[2];          // bit storage, ping-pong
    uint32_t *fit[2];          // fitness, ping-pong
    uint32_t *state;           // kFusedStateWords words, zeroed before each launch
    unsigned long long *tmask; // [ntiles] (F < T) | (F == T) << 32 per tile
    const uint32_t *perm;      // [ngen][2N] survivor orders of the chunk
    unsigned long long *traj;  // [traj_cap] best keys (F << 32 | slot)
    uint32_t *gen_dev;         // generation counter: read at start, advanced at exit
    int8_t *gram;              // incremental mode: [P][dpad] tiled half-Gram (common.cuh), or null
    uint32_t *gidx[2];         // incremental mode: slot -> Gram buffer, ping-pong with pop
    unsigned long long *cw;    // probabilistic selection: in-tile weight prefixes [ntiles][32]
    int32_t dpad;              // bytes per Gram buffer (64 per tile)
    int32_t m, W, NC, NR, kind, traj_cap;
    int32_t nch;                 // chunks per column of the warp-level Gram (m > 32; autotuned)
    int32_t tpp;                 // threads per pair of the m <= 32 build, 2 or 4 (autotuned)
    int32_t shared_mut;          // mutation method 1: every offspring draws from stream index 2N
    int64_t N;
    uint32_t seed, pop_id;
    uint32_t tile_base, ntiles;  // tiles of 32 slots in the joint tile space
    uint32_t work_base;          // m <= 32: first thread slot; m > 32: first pair
};

struct FusedParams {
    FusedPop p[kMaxPops];
    int32_t npop;
    uint32_t total_tiles;
    uint32_t thread_slots;   // joint space of m <= 32 populations, 2 threads per pair, padded to 32
    uint32_t warp_items;     // joint offspring space of m > 32 populations (one warp item each)
    int32_t ngen;            // generations to run
    int32_t stop_at_zero;    // stop after a generation whose best fitness (population 0) is 0
    int32_t src;             // ping-pong buffer holding the current population
    int32_t warp_buf_words;  // shared words per warp for m > 32 populations
    int32_t inc_ring;        // 16-byte slots per warp of the incremental copy ring (0: no incremental population)
    int32_t psel;            // probabilistic selection (every population), else truncation
    uint32_t *bar;           // grid-barrier counter (zeroed before the launch)
    uint32_t *err;           // device error word
    int32_t *done;           // generations completed
};

size_t fused_smem_bytes(const FusedParams &p);
// Dynamic shared memory a block of the persistent kernel may take on the
// current device (opt-in maximum less the kernel's static shared memory).
size_t fused_smem_limit();
// Sets p.inc_ring: the largest copy ring (up to one offspring's phase-1
// copies) that keeps the block's shared memory within the device limit.
void fused_plan_ring(FusedParams &p);
cudaError_t fused_grid(size_t smem, int *grid);
cudaError_t launch_fused(const FusedParams &p, int grid, size_t smem, cudaStream_t s);

} // namespace hadga
