// k_tc.cu -- tcgen05 (5th-generation tensor core) Gram + fitness paths for
// FP8 e4m3 and BF16 storage.  Not built yet in this revision: the entry
// points report "not supported" so callers get GA_EUNSUPPORTED.
#include "common.cuh"
#include "kernels.cuh"

namespace hadga {

bool fitness_tc_supported(int storage, int m)
{
    (void)storage;
    (void)m;
    return false;
}

cudaError_t launch_fitness_tc(const void *pop, int storage, int m, int64_t first, int64_t count, int kind,
                              uint32_t *fit, uint32_t *err, cudaStream_t s)
{
    (void)pop; (void)storage; (void)m; (void)first; (void)count; (void)kind; (void)fit; (void)err; (void)s;
    return cudaErrorNotSupported;
}

} // namespace hadga
