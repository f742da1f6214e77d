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
cudaError_t launch_mutate(void *pop, int storage, int m, int64_t N, int NC, int NR, uint32_t seed, uint32_t pop_id,
                          uint32_t gen, cudaStream_t s);
// Least (F << 32 | slot) of fit[0, P) into *out (which is first set to ~0).
cudaError_t launch_best(const uint32_t *fit, int64_t P, unsigned long long *out, cudaStream_t s);
cudaError_t launch_convert(const void *src, int src_storage, void *dst, int dst_storage, int m, int64_t P,
                           cudaStream_t s);

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
};
// Selection of generation `gen`: leaves in scratch_pop[0, 2N) / scratch_fit the
// parents in placement order (matrix bytes per slot = mat_bytes).
cudaError_t launch_select(const void *pop, const uint32_t *fit, int64_t N, size_t mat_bytes, uint32_t seed,
                          uint32_t pop_id, uint32_t gen, const SelWork &w, void *scratch_pop, uint32_t *scratch_fit,
                          cudaStream_t s);
// Survivor orders pi of `ngen` consecutive generations gen0.. into out[ngen][n]
// (n <= kPermSmemMax), one block per generation.
cudaError_t launch_perm_table(uint32_t n, uint32_t seed, uint32_t pop_id, uint32_t gen0, int ngen, uint32_t *out,
                              cudaStream_t s);
int perm_global_bits(uint32_t n);

// ---- fused persistent generation kernel (k_fused.cu) -------------------------
struct FusedPop {
    uint32_t *pop[2];          // bit storage, ping-pong
    uint32_t *fit[2];
    uint32_t *hist[2];         // level-0 histograms, ping-pong by generation
    uint32_t *hist_ref;        // refinement histogram
    unsigned long long *tmask; // [tiles]
    const uint32_t *perm;      // [chunk][2N]
    unsigned long long *traj;  // [traj_cap]
    uint32_t *orv;             // [2] OR of all fitness values, by generation parity
    uint32_t *cap;             // [2] histogram cap (threshold of the previous generation)
    int32_t m, W, NC, NR, kind, traj_cap;
    int64_t N;
    uint32_t seed, pop_id;
    uint32_t tile_base;        // first tile of this population in the joint tile space
    uint32_t pair_base;        // first pair-chunk slot in the joint pair space (multiple of 32)
};

struct FusedArgs {
    const FusedPop *pops;      // device array
    int32_t npop;
    uint32_t total_tiles;
    uint32_t total_pair_slots; // joint pair space (each population padded to 32)
    uint32_t gen0;             // generation before the chunk
    int32_t ngen;              // generations in this chunk
    int32_t stop_at_zero;
    int32_t src;               // which ping-pong buffer holds the current state
    uint32_t *bar;
    uint32_t *err;
    int32_t *done;             // generations completed (device)
};

cudaError_t launch_fused_prepare(const FusedArgs &a, int npop_host, const FusedPop *pops_host, cudaStream_t s);
cudaError_t launch_fused(const FusedArgs &a, int blocks, int threads, size_t smem, cudaStream_t s);
cudaError_t fused_occupancy(int threads, size_t smem, int *blocks_per_sm);
size_t fused_smem_bytes(uint32_t total_tiles, int threads);

} // namespace hadga
