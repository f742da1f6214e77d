// k_debug.cu -- test-only exports: the bounded device waits driven to their
// limit, on purpose and without any fault.
//
// The kernels below call the very wait functions the generation kernels use
// (grid_barrier of the persistent kernel, mbar_wait of the tensor-core and
// bulk-copy pipelines) on a target that can never be met: a grid barrier
// expecting one more arrival than there are blocks, an mbarrier nobody
// arrives on.  With a short budget the wait gives up, records ERR_TIMEOUT in
// the error word and the kernel returns normally; the host reads the word
// after a stream synchronisation, exactly as ga_sync does.  No trap, no
// assert, no invalid address: the context stays usable.
#include "hadga.h"
#include "common.cuh"
#include "kernels.cuh"

namespace hadga {
namespace {

__global__ void k_debug_grid_wait(uint32_t *bar, uint32_t *err, unsigned long long budget_ns)
{
    uint32_t epoch = 0;
    // nblocks + 1 arrivals expected: the barrier cannot complete
    grid_barrier(bar, gridDim.x + 1u, epoch, err, budget_ns);
}

__global__ void k_debug_mbar_wait(uint32_t *err, unsigned long long budget_ns)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // phase 0 needs one arrival that never comes
    if (threadIdx.x == 0)
        mbar_wait(&bar, 0u, err, budget_ns);
    __syncthreads();
}

} // namespace
} // namespace hadga

using namespace hadga;

extern "C" ga_status ga_debug_wait_timeout(int32_t which, uint32_t budget_us, uint32_t *err_out, void *stream)
{
    if (which != 0 && which != 1)
        return (set_thread_error("ga_debug_wait_timeout: which must be 0 (grid barrier) or 1 (mbarrier)"), GA_EINVAL);
    if (budget_us < 1u || budget_us > 1000000u)
        return (set_thread_error("ga_debug_wait_timeout: budget_us must lie in [1, 1000000]"), GA_EINVAL);
    if (!err_out)
        return (set_thread_error("ga_debug_wait_timeout: err_out is NULL"), GA_EINVAL);
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t *mem = nullptr;  // [0] barrier counter, [1] error word
    cudaError_t e = cudaMalloc(&mem, 2 * sizeof(uint32_t));
    if (e == cudaSuccess)
        e = cudaMemsetAsync(mem, 0, 2 * sizeof(uint32_t), s);
    const unsigned long long ns = (unsigned long long)budget_us * 1000ull;
    if (e == cudaSuccess) {
        if (which == 0) {
            // two co-resident blocks (cooperative launch), as in the persistent kernel
            uint32_t *bar = mem, *err = mem + 1;
            unsigned long long budget = ns;
            void *args[] = {(void *)&bar, (void *)&err, (void *)&budget};
            e = cudaLaunchCooperativeKernel((const void *)k_debug_grid_wait, dim3(2), dim3(64), args, 0, s);
        } else {
            k_debug_mbar_wait<<<1, 32, 0, s>>>(mem + 1, ns);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess)
            note_launches(1);
    }
    uint32_t w = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&w, mem + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (mem)
        cudaFree(mem);
    if (e != cudaSuccess) {
        set_thread_error(cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? GA_ENOMEM : GA_ECUDA;
    }
    *err_out = w;
    if (w & ERR_TIMEOUT) {
        set_thread_error("a bounded device wait exceeded its budget (device error word has ERR_TIMEOUT)");
        return GA_ETIMEOUT;
    }
    if (w) {
        set_thread_error("device-side check failed");
        return GA_ECUDA;
    }
    return GA_OK;
}
