// k_gram_real.cu -- batched Gram G_b = Q_b^T Q_b of B real m x m matrices in
// FP64 or FP32 on the CUDA cores: the speed comparison of Sec. 2 (Table 1,
// N = 10,000 random 100 x 100 float64 matrices, each multiplied by its own
// transpose).  It is not a step of the GA.
//
// G = sum over rows r of q_r^T q_r (q_r the r-th row of Q), so a block streams
// its matrix through shared memory a chunk of rows at a time (cp.async into
// two buffers, the next chunk in flight while one is multiplied), and each
// thread accumulates an R x R tile of G in registers.  The column indices are
// split into nt groups of R; tiles (ti, tj) with ti <= tj cover the upper
// triangle of the group grid, and each tile is written once as itself and
// once as its mirror image (G is symmetric), so a block does about
// (m^3 + m^2 R) / 2 multiply-adds (m rounded up to a multiple of R) instead
// of the m^3 of a general matrix product.  Entry (i, j) is the sum over
// r = 0 .. m-1 in ascending order, one fused multiply-add per term, in the
// input's own precision.
//
// Group g holds two runs of R/2 columns (16 bytes each): g R/2 .. g R/2 +
// R/2 - 1 and H + g R/2 .. H + g R/2 + R/2 - 1, with H = nt R/2.  Threads of a
// warp hold consecutive groups, so each 16-byte shared-memory load of a warp
// reads one contiguous span (no bank conflicts), where a run of R contiguous
// columns per thread would read every other 16 bytes.
#include "common.cuh"
#include "kernels.cuh"

namespace hadga {
namespace {

// Register tile edge: 4 x 4 in FP64 (the FMA pipe is the bound at any
// tile), 8 x 8 in FP32 (four shared-memory vector loads per 64 FMAs).
// Threads per block at most, and the register budget those leave.
template <typename T>
struct RealTile {
    static constexpr int R = sizeof(T) == 8 ? 4 : 8;
    static constexpr int kMaxThreads = sizeof(T) == 8 ? 512 : 256;
    static constexpr int kMinBlocks = sizeof(T) == 8 ? 1 : 2;  // FP32: <= 128 registers
    static constexpr int kChunkBytes = sizeof(T) == 8 ? 24576 : 16384;  // one of the two row buffers
};

// 16 bytes (R/2 elements) from shared memory.
__device__ __forceinline__ void ld16(const double *p, double *v)
{
    const double2 x = *reinterpret_cast<const double2 *>(p);
    v[0] = x.x;
    v[1] = x.y;
}

__device__ __forceinline__ void ld16(const float *p, float *v)
{
    const float4 x = *reinterpret_cast<const float4 *>(p);
    v[0] = x.x;
    v[1] = x.y;
    v[2] = x.z;
    v[3] = x.w;
}

// 16 bytes (R/2 elements) to global memory.
__device__ __forceinline__ void st16(double *p, const double *v)
{
    *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
}

__device__ __forceinline__ void st16(float *p, const float *v)
{
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

// Column (or row) index of element e of group g: e < R/2 in the first run,
// the rest in the second run H further on.
template <int R>
__device__ __forceinline__ int group_index(int g, int e, int H)
{
    return (e < R / 2 ? 0 : H) + g * (R / 2) + (e % (R / 2));
}

// Tile u of the row-major enumeration of the upper triangle of an nt x nt
// tile grid -> (ti, tj), ti <= tj.
__device__ __forceinline__ void upper_tile(int u, int nt, int &ti, int &tj)
{
    int i = 0;
    while (u >= nt - i) {
        u -= nt - i;
        ++i;
    }
    ti = i;
    tj = i + u;
}

// One chunk step of a block: matrix b, tile pass u0 (tiles u0 .. u0 +
// blockDim - 1 of the upper triangle), rows k0 .. k0 + kc - 1 of Q.
struct RealStep {
    int64_t b;
    int u0;
    int k0;
};

__device__ __forceinline__ bool real_next(RealStep &st, int64_t B, int U, int nthr, int m, int kc_max)
{
    st.k0 += kc_max;
    if (st.k0 < m)
        return true;
    st.k0 = 0;
    st.u0 += nthr;
    if (st.u0 < U)
        return true;
    st.u0 = 0;
    st.b += gridDim.x;
    return st.b < B;
}

// Issues the asynchronous copies of the rows of step `st` into `buf` (row
// pitch sp): 16-byte copies when a row of Q is a whole number of 16-byte
// units, element copies otherwise.
template <typename T>
__device__ __forceinline__ void real_issue(const T *q, int m, int sp, int kc_max, const RealStep &st, T *buf,
                                           bool vec_rows)
{
    const int kc = min(kc_max, m - st.k0);
    const T *src = q + ((size_t)st.b * m + st.k0) * m;
    if (vec_rows) {
        constexpr int E = 16 / (int)sizeof(T);  // elements per 16-byte unit
        const int upr = m / E;
        for (int e = threadIdx.x; e < kc * upr; e += blockDim.x) {
            const int r = e / upr, x = e - r * upr;
            cp_async16(buf + r * sp + x * E, src + (size_t)r * m + x * E);
        }
    } else {
        for (int e = threadIdx.x; e < kc * m; e += blockDim.x) {
            const int r = e / m, c = e - r * m;
            cp_async_small<(int)sizeof(T)>(buf + r * sp + c, src + e);
        }
    }
}

// One block per matrix at a time (grid-stride over the batch).  Shared
// memory holds two buffers of `kc_max` rows of Q with a row pitch of
// sp = nt * R elements: the next chunk (of this matrix, or of the block's
// next one) is copied in while the current one is multiplied.  Columns
// m .. sp-1 are zero so that edge tiles need no bounds checks in the inner
// loop.
template <typename T>
__global__ void __launch_bounds__(RealTile<T>::kMaxThreads, RealTile<T>::kMinBlocks)
    k_gram_real(const T *__restrict__ q, T *__restrict__ g, int m, int64_t B, int kc_max)
{
    extern __shared__ __align__(16) unsigned char real_smem[];
    constexpr int R = RealTile<T>::R, R2 = R / 2;
    const int nt = (m + R - 1) / R, sp = nt * R, H = nt * R2;
    const int U = nt * (nt + 1) / 2;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const bool vec_rows = (m * (int)sizeof(T)) % 16 == 0;
    T *const buf0 = reinterpret_cast<T *>(real_smem);
    const int buf_elems = kc_max * sp;  // second buffer at buf0 + buf_elems

    RealStep cur{(int64_t)blockIdx.x, 0, 0};
    if (cur.b >= B)
        return;
    if (sp > m)  // zero padding columns of both buffers once; copies never write them
        for (int e = tid; e < 2 * kc_max * (sp - m); e += nthr)
            buf0[(e / (sp - m)) * sp + m + e % (sp - m)] = T(0);
    real_issue<T>(q, m, sp, kc_max, cur, buf0, vec_rows);
    cp_async_commit();
    RealStep nxt = cur;
    bool has_next = real_next(nxt, B, U, nthr, m, kc_max);

    int ti = 0, tj = 0;
    bool active = tid < U;
    if (active)
        upper_tile(tid, nt, ti, tj);
    T acc[R][R];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < R; ++c)
            acc[r][c] = T(0);

    for (int parity = 0;; parity ^= 1) {
        if (has_next)
            real_issue<T>(q, m, sp, kc_max, nxt, buf0 + (parity ^ 1) * buf_elems, vec_rows);
        cp_async_commit();
        cp_async_wait_group<1>();  // the current chunk has landed (this thread's copies)
        __syncthreads();           // ... and every thread's
        const int kc = min(kc_max, m - cur.k0);
        if (active) {
            const T *pa = buf0 + parity * buf_elems + ti * R2, *pb = buf0 + parity * buf_elems + tj * R2;
#pragma unroll 2
            for (int kk = 0; kk < kc; ++kk) {
                T a[R], v[R];
                ld16(pa + kk * sp, a);
                ld16(pa + kk * sp + H, a + R2);
                ld16(pb + kk * sp, v);
                ld16(pb + kk * sp + H, v + R2);
#pragma unroll
                for (int r = 0; r < R; ++r)
#pragma unroll
                    for (int c = 0; c < R; ++c)
                        acc[r][c] = fma(a[r], v[c], acc[r][c]);
            }
        }
        if (cur.k0 + kc >= m) {  // end of a tile pass: write the tiles
            if (active) {
                T *gb = g + (size_t)cur.b * m * m;
                if (vec_rows) {  // 16-byte runs, each wholly inside or outside the matrix
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const int i = group_index<R>(ti, r, H);
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int j = h * H + tj * R2;
                            if (i < m && j < m)
                                st16(gb + (size_t)i * m + j, &acc[r][h * R2]);
                        }
                    }
                    if (ti != tj)
#pragma unroll
                        for (int c = 0; c < R; ++c) {
                            const int j = group_index<R>(tj, c, H);
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                const int i = h * H + ti * R2;
                                T col[R2];
#pragma unroll
                                for (int e = 0; e < R2; ++e)
                                    col[e] = acc[h * R2 + e][c];
                                if (i < m && j < m)
                                    st16(gb + (size_t)j * m + i, col);
                            }
                        }
                } else {
#pragma unroll
                    for (int r = 0; r < R; ++r)
#pragma unroll
                        for (int c = 0; c < R; ++c) {
                            const int i = group_index<R>(ti, r, H), j = group_index<R>(tj, c, H);
                            if (i < m && j < m) {
                                gb[(size_t)i * m + j] = acc[r][c];
                                if (ti != tj)
                                    gb[(size_t)j * m + i] = acc[r][c];
                            }
                        }
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int c = 0; c < R; ++c)
                    acc[r][c] = T(0);
        }
        __syncthreads();  // the buffer just read is refilled by the next trip
        if (!has_next)
            break;
        cur = nxt;
        has_next = real_next(nxt, B, U, nthr, m, kc_max);
        if (cur.k0 == 0) {
            const int u = cur.u0 + tid;
            active = u < U;
            if (active)
                upper_tile(u, nt, ti, tj);
        }
    }
    cp_async_wait_group<0>();
}

template <typename T>
void real_shape(int m, int &threads, int &kc, size_t &smem)
{
    constexpr int R = RealTile<T>::R, tmax = RealTile<T>::kMaxThreads;
    const int nt = (m + R - 1) / R, sp = nt * R;
    const int U = nt * (nt + 1) / 2;
    const int passes = (U + tmax - 1) / tmax;
    threads = (((U + passes - 1) / passes + 31) / 32) * 32;
    kc = RealTile<T>::kChunkBytes / (sp * (int)sizeof(T));
    if (kc > m)
        kc = m;
    if (kc < 1)
        kc = 1;
    smem = 2 * (size_t)kc * sp * sizeof(T);
}

template <typename T>
cudaError_t launch_real(const T *q, T *g, int m, int64_t B, cudaStream_t s)
{
    static bool carveout_set = false;  // prefer shared memory over L1 (several blocks per SM)
    if (!carveout_set) {
        cudaFuncSetAttribute(k_gram_real<T>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
        carveout_set = true;
    }
    int threads = 0, kc = 0;
    size_t smem = 0;
    real_shape<T>(m, threads, kc, smem);
    const unsigned grid = (unsigned)(B < (int64_t)0x7fffffff ? B : (int64_t)0x7fffffff);
    k_gram_real<T><<<grid, threads, smem, s>>>(q, g, m, B, kc);
    note_launches(1);
    return cudaGetLastError();
}

} // namespace

// Threads per block, rows per shared-memory chunk and dynamic shared memory
// of the batched real Gram at order m for an element of `elem` bytes: the
// upper tiles are dealt evenly to the fewest passes of at most
// RealTile<T>::kMaxThreads threads.
void gram_real_shape(int m, int elem, int &threads, int &kc, size_t &smem)
{
    if (elem == 8)
        real_shape<double>(m, threads, kc, smem);
    else
        real_shape<float>(m, threads, kc, smem);
}

cudaError_t launch_gram_real(const void *q, void *g, int f64, int m, int64_t B, cudaStream_t s)
{
    if (B <= 0)
        return cudaSuccess;
    if (f64)
        return launch_real<double>(static_cast<const double *>(q), static_cast<double *>(g), m, B, s);
    return launch_real<float>(static_cast<const float *>(q), static_cast<float *>(g), m, B, s);
}

} // namespace hadga
