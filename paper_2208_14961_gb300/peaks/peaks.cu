// peaks.cu -- throughput microbenchmarks of the instruction classes the
// Gram paths use on this GPU (not part of libhadga): 32-bit population count,
// 4-way byte dot product (dp4a) and warp-level int8 tensor-core MMA.
// Each kernel runs long dependent-free chains per thread and returns a
// checksum so the compiler keeps the work; the host times it with events.
#include <cstdint>
#include <cuda_runtime.h>

namespace {

__global__ void k_popc(uint32_t *out, int iters)
{
    uint32_t x[8], acc[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        x[i] = threadIdx.x * 2654435761u + i * 40503u + blockIdx.x;
        acc[i] = 0;
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            acc[i] += __popc(x[i]);
            x[i] = x[i] * 1664525u + 1013904223u;
        }
    }
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i)
        s += acc[i];
    if (s == 0x12345678u)
        out[0] = s;
}

__global__ void k_popc_only(uint32_t *out, int iters)
{
    uint32_t x[16], acc[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        x[i] = threadIdx.x * 2654435761u + i * 40503u + blockIdx.x;
        acc[i] = 0;
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 16; ++i)
            acc[i] ^= __popc(x[i] ^ acc[i]);
    }
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i)
        s += acc[i];
    if (s == 0x12345678u)
        out[0] = s;
}

__global__ void k_dp4a(uint32_t *out, int iters)
{
    int a[8], acc[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        a[i] = (int)(threadIdx.x * 2654435761u + i);
        acc[i] = i;
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i)
            acc[i] = __dp4a(a[i], a[(i + 1) & 7], acc[i]);
    }
    int s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i)
        s += acc[i];
    if (s == 0x12345678)
        out[0] = (uint32_t)s;
}

__global__ void k_imma(uint32_t *out, int iters)
{
    uint32_t a[4] = {threadIdx.x, threadIdx.x * 3u, threadIdx.x * 5u, threadIdx.x * 7u};
    uint32_t b[2] = {threadIdx.x * 11u, threadIdx.x * 13u};
    int d[4][4] = {};
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 "
                         "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                         : "+r"(d[j][0]), "+r"(d[j][1]), "+r"(d[j][2]), "+r"(d[j][3])
                         : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
    int s = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j)
        s += d[j][0] + d[j][1] + d[j][2] + d[j][3];
    if (s == 0x12345678)
        out[0] = (uint32_t)s;
}

} // namespace

// kind: 0 popc (mixed with an integer update), 1 popc chain, 2 dp4a, 3 mma.sync s8.
// Returns the operations per second (popc / dp4a instructions per lane, or
// int8 multiply-adds for the MMA) measured over `iters` loop trips.
extern "C" double peak_rate(int kind, int iters)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint32_t *out = nullptr;
    if (cudaMalloc(&out, 4) != cudaSuccess)
        return -1.0;
    const int blocks = sms * 8, threads = 256;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    double ops_per_thread = 0.0;
    for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(a);
        switch (kind) {
        case 0: k_popc<<<blocks, threads>>>(out, iters); ops_per_thread = 8.0 * iters; break;
        case 1: k_popc_only<<<blocks, threads>>>(out, iters); ops_per_thread = 16.0 * iters; break;
        case 2: k_dp4a<<<blocks, threads>>>(out, iters); ops_per_thread = 8.0 * iters; break;
        default: k_imma<<<blocks, threads>>>(out, iters); ops_per_thread = 4.0 * iters * 4096.0 / 32.0; break;
        }
        cudaEventRecord(b);
    }
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(out);
    if (cudaGetLastError() != cudaSuccess || ms <= 0.f)
        return -1.0;
    return ops_per_thread * blocks * threads / (ms * 1e-3);
}
