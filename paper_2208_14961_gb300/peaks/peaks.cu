// peaks.cu -- throughput microbenchmarks of the instruction classes the
// Gram paths use on this GPU (not part of libhadga): 32-bit population count,
// 4-way byte dot product (dp4a), 32-bit integer multiply-add, warp-level int8
// and e4m3 tensor-core MMA, FP64 and FP32 fused multiply-add, L2 read
// bandwidth and the latency of the grid barrier of the fused generation kernel.
// Each kernel runs long dependent-free chains per thread and returns a
// checksum so the compiler keeps the work; the host times it with events.
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

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

__global__ void k_imad(uint32_t *out, int iters)
{
    uint32_t x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
        x[i] = threadIdx.x * 2654435761u + i;
    for (int it = 0; it < iters; ++it) {
        // each multiplier depends on the previous step (no closed form)
#pragma unroll
        for (int i = 0; i < 8; ++i)
            x[i] = x[i] * (x[(i + 1) & 7] | 1u) + (uint32_t)it;
    }
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i)
        s += x[i];
    if (s == 0x12345678u)
        out[0] = s;
}

__global__ void k_mma_e4m3(uint32_t *out, int iters)
{
    uint32_t a[4] = {0x38383838u, 0xB8383838u, 0x3838B838u, 0x38B83838u};
    uint32_t b[2] = {0x383838B8u, 0x38383838u};
    float d[4][4] = {};
    for (int it = 0; it < iters; ++it) {
        // operands change every trip (sign bits of +-1 in e4m3)
        a[it & 3] ^= 0x80000000u;
        b[it & 1] ^= 0x00800000u;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            asm volatile("mma.sync.aligned.m16n8k32.row.col.f32.e4m3.e4m3.f32 "
                         "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                         : "+f"(d[j][0]), "+f"(d[j][1]), "+f"(d[j][2]), "+f"(d[j][3])
                         : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j)
        s += d[j][0] + d[j][1] + d[j][2] + d[j][3];
    if (s == 1234.5f)
        out[0] = 1u;
}

// Fused multiply-adds in T (double or float): 8 independent chains a thread.
template <typename T>
__global__ void k_fma(uint32_t *out, int iters)
{
    T x[8];
    const T c = T(0.999755859375), d = T(0.000244140625) * T(threadIdx.x & 7);
#pragma unroll
    for (int i = 0; i < 8; ++i)
        x[i] = T(threadIdx.x + i) * T(0.0009765625);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i)
            x[i] = fma(x[i], c, d);
    }
    T s = T(0);
#pragma unroll
    for (int i = 0; i < 8; ++i)
        s += x[i];
    if (s == T(1234.5))
        out[0] = 1u;
}

// Reads `n4` 16-byte words of `buf` (small enough to stay in L2) `iters`
// times through L2 (ld.global.cg), grid-stride.
__global__ void k_l2_read(const uint4 *__restrict__ buf, size_t n4, int iters, uint32_t *out)
{
    uint32_t acc = 0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (int it = 0; it < iters; ++it)
        for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n4; e += stride) {
            const uint4 v = __ldcg(buf + e);
            acc ^= v.x ^ v.y ^ v.z ^ v.w;
        }
    if (acc == 0x12345678u)
        out[0] = acc;
}

// `iters` grid-wide barriers of the fused kernel's kind (one block per SM,
// 512 threads, cooperative launch).
__global__ void __launch_bounds__(512, 1) k_grid_barriers(uint32_t *bar, uint32_t *err, int iters)
{
    uint32_t epoch = 0;
    for (int it = 0; it < iters; ++it)
        if (!hadga::grid_barrier(bar, gridDim.x, epoch, err))
            return;
}

static double l2_read_rate(int sms, int iters)
{
    const size_t bytes = (size_t)64 << 20;  // half of the L2
    uint4 *buf = nullptr;
    uint32_t *out = nullptr;
    if (cudaMalloc(&buf, bytes) != cudaSuccess)
        return -1.0;
    if (cudaMalloc(&out, 4) != cudaSuccess) {
        cudaFree(buf);
        return -1.0;
    }
    cudaMemset(buf, 1, bytes);
    const int it = iters / 64 > 0 ? iters / 64 : 1;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    k_l2_read<<<sms * 4, 512>>>(buf, bytes / 16, 1, out);  // warm the L2
    cudaEventRecord(a);
    k_l2_read<<<sms * 4, 512>>>(buf, bytes / 16, it, out);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(buf);
    cudaFree(out);
    if (cudaGetLastError() != cudaSuccess || ms <= 0.f)
        return -1.0;
    return (double)bytes * it / (ms * 1e-3);
}

static double grid_barrier_rate(int sms, int iters)
{
    uint32_t *w = nullptr;
    if (cudaMalloc(&w, 8) != cudaSuccess)
        return -1.0;
    cudaMemset(w, 0, 8);
    uint32_t *bar = w, *err = w + 1;
    int n = iters;
    void *args[] = {&bar, &err, &n};
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a);
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)k_grid_barriers, dim3(sms), dim3(512), args, 0, 0);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    uint32_t h_err = 0;
    cudaMemcpy(&h_err, err, 4, cudaMemcpyDeviceToHost);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(w);
    if (e != cudaSuccess || h_err != 0u || cudaGetLastError() != cudaSuccess || ms <= 0.f)
        return -1.0;
    return iters / (ms * 1e-3);
}

} // namespace

// kind: 0 popc (mixed with an integer update), 1 popc chain, 2 dp4a, 3 mma.sync s8,
// 4 IMAD, 5 mma.sync e4m3 (multiply-adds), 6 L2 read bytes, 7 grid barriers,
// 8 FP64 fused multiply-adds, 9 FP32 fused multiply-adds.
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
    if (kind == 6 || kind == 7) {
        cudaFree(out);
        return kind == 6 ? l2_read_rate(sms, iters) : grid_barrier_rate(sms, iters);
    }
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
        case 4: k_imad<<<blocks, threads>>>(out, iters); ops_per_thread = 8.0 * iters; break;
        case 8: k_fma<double><<<blocks, threads>>>(out, iters); ops_per_thread = 8.0 * iters; break;
        case 9: k_fma<float><<<blocks, threads>>>(out, iters); ops_per_thread = 8.0 * iters; break;
        case 5: k_mma_e4m3<<<blocks, threads>>>(out, iters); ops_per_thread = 4.0 * iters * 4096.0 / 32.0; break;
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
