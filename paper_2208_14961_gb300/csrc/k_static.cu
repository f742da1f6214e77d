// k_static.cu -- ga_select_static: the selection step (truncation selection
// and random placement of the survivors) without any device allocation.
//
// Some callers cannot call cudaMalloc while they run this step: code that
// executes inside a framework's execution hook where device memory must not
// be allocated (plugin enqueue functions with a fixed workspace, pooled
// allocators that forbid out-of-pool allocations), or code on a hot path
// where an allocation would implicitly synchronise the device.  For them the
// scratch of the selection lives in one file-scope device array of fixed
// size, held by every GPU that loads the library's device code until the
// process exits.  Under CUDA's default lazy module loading that code (and
// the array with it) is loaded on a device at its first use -- the first
// call of this entry point or of any other kernel of this file -- and that
// load can itself take device memory, so one warm-up call per device must
// come before any region that forbids allocation or stream capture.  The
// device address found by that first call is kept per device ordinal; it
// belongs to the device's current (primary) context and must not be used
// after that context is destroyed (cudaDeviceReset), which this library
// cannot detect.
#include <mutex>
#include <string>

#include "common.cuh"
#include "hadga.h"
#include "kernels.cuh"

namespace hadga {
namespace {

// Largest N the allocation-free selection accepts (P = 4N <= 32768).
constexpr int64_t kStaticMaxN = 8192;
// Scratch layout (bytes): histogram 2048 words, selection state, the device
// error word (in a 256-byte block of its own, at a fixed offset), then per tile
// (P/32 tiles) an 8-byte mask pair and two 4-byte words and the survivor order
// (2N words).
constexpr size_t kStaticHistBytes = 2048 * 4;
constexpr size_t kStaticStateBytes = 256;
constexpr size_t kStaticErrOff = kStaticHistBytes + kStaticStateBytes;
constexpr size_t kStaticTiles = (size_t)(4 * kStaticMaxN) / 32;
constexpr size_t kStaticScratchBytes =
    kStaticHistBytes + kStaticStateBytes + kStaticTiles * (8 + 4 + 4) + (size_t)(2 * kStaticMaxN) * 4 + 256;

static __device__ __align__(256) unsigned char g_select_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_scratch_addr[kMaxDevices] = {};

ga_status fail(ga_status st, const char *msg)
{
    set_thread_error(msg);  // reported by ga_last_error(NULL)
    return st;
}

// The current device's address of the scratch array (its host-side name is
// only a stand-in), looked up once per device with that device current.
ga_status scratch_base(const char *who, unsigned char **base)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(GA_ECUDA, (std::string(who) + ": no usable current device").c_str());
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_select_scratch);
        if (e != cudaSuccess || !ptr)
            return fail(GA_ECUDA, (std::string(who) + ": cudaGetSymbolAddress of the scratch array failed").c_str());
        g_scratch_addr[dev] = ptr;
    }
    *base = (unsigned char *)g_scratch_addr[dev];
    return GA_OK;
}

} // namespace
} // namespace hadga

using namespace hadga;

extern "C" ga_status ga_select_static(const void *pop_in, const uint32_t *fit_in, void *parents_out,
                                      uint32_t *parent_fit_out, int32_t storage, int32_t m, int64_t N, uint32_t seed,
                                      uint32_t pop_id, uint32_t gen, void *stream)
{
    if (!pop_in || !fit_in || !parents_out || !parent_fit_out)
        return fail(GA_EINVAL, "ga_select_static: NULL buffer");
    if (m < 4 || m > kMaxM || (m & 3) || (storage != ST_INT8 && storage != ST_BITS))
        return fail(GA_EINVAL, "ga_select_static: m must be a multiple of 4 in [4, 256], storage INT8 or BITS");
    if (N < 1 || N > kStaticMaxN)
        return fail(GA_EINVAL, "ga_select_static: N must lie in [1, 8192] (P <= 32768): the fixed scratch array "
                               "holds no more");
    if ((((uintptr_t)pop_in) | ((uintptr_t)fit_in) | ((uintptr_t)parents_out) | ((uintptr_t)parent_fit_out)) & 15u)
        return fail(GA_EINVAL, "ga_select_static: buffers must be 16-byte aligned");
    const size_t mat = matrix_bytes(storage, m);
    // every output is written while the inputs are still read (the gather
    // reads fit_in[src] for any src while parent_fit_out[p] is written), so
    // no output may share bytes with an input or with the other output
    struct Span {
        uintptr_t lo, hi;
        const char *name;
    };
    const Span in[2] = {{(uintptr_t)pop_in, (uintptr_t)pop_in + (size_t)(4 * N) * mat, "pop_in"},
                        {(uintptr_t)fit_in, (uintptr_t)fit_in + (size_t)(4 * N) * 4u, "fit_in"}};
    const Span out[2] = {{(uintptr_t)parents_out, (uintptr_t)parents_out + (size_t)(2 * N) * mat, "parents_out"},
                         {(uintptr_t)parent_fit_out, (uintptr_t)parent_fit_out + (size_t)(2 * N) * 4u,
                          "parent_fit_out"}};
    auto overlap = [](const Span &a, const Span &b) { return a.lo < b.hi && b.lo < a.hi; };
    for (const Span &o : out)
        for (const Span &i : in)
            if (overlap(o, i)) {
                set_thread_error((std::string("ga_select_static: ") + o.name + " must not overlap " + i.name).c_str());
                return GA_EINVAL;
            }
    if (overlap(out[0], out[1]))
        return fail(GA_EINVAL, "ga_select_static: parents_out must not overlap parent_fit_out");

    unsigned char *base = nullptr;
    const ga_status st = scratch_base("ga_select_static", &base);
    if (st != GA_OK)
        return st;

    const int64_t tiles = (4 * N + 31) / 32;
    SelWork w{};
    size_t off = 0;
    w.hist = (uint32_t *)(base + off);
    off += kStaticHistBytes;
    w.state = (SelState *)(base + off);
    off += kStaticStateBytes;
    w.err = (uint32_t *)(base + off);
    off += 256;
    w.tmask = (unsigned long long *)(base + off);
    off += (size_t)tiles * 8;
    w.survmask = (uint32_t *)(base + off);
    off += (size_t)tiles * 4;
    w.survbefore = (uint32_t *)(base + off);
    off += (size_t)tiles * 4;
    w.perm = (uint32_t *)(base + off);
    off += (size_t)(2 * N) * 4;
    w.perm_keys = nullptr;  // 2N <= 16384 always takes the shared-memory sort
    w.perm_cnt = nullptr;

    cudaStream_t s = (cudaStream_t)stream;
    // the array keeps the previous call's contents: clear what must start at 0
    cudaError_t e = cudaMemsetAsync(w.hist, 0, kStaticHistBytes + kStaticStateBytes, s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(w.err, 0, 4, s);
    if (e == cudaSuccess)
        e = launch_select(pop_in, fit_in, N, mat, seed, pop_id, gen, w, parents_out, parent_fit_out, s);
    if (e != cudaSuccess)
        return fail(GA_ECUDA, cudaGetErrorString(e));
    return GA_OK;
}

extern "C" ga_status ga_select_static_error(uint32_t *err_out, void *stream)
{
    if (!err_out)
        return fail(GA_EINVAL, "ga_select_static_error: NULL err_out");
    unsigned char *base = nullptr;
    const ga_status st = scratch_base("ga_select_static_error", &base);
    if (st != GA_OK)
        return st;
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t word = 0;
    cudaError_t e = cudaMemcpyAsync(&word, base + kStaticErrOff, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return fail(GA_ECUDA, cudaGetErrorString(e));
    *err_out = word;
    return GA_OK;
}
