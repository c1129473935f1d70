// residual_noalloc.cu -- ||b - A x|| and ||b|| of a caller-held device CSR
// without allocating anything.
//
// Who needs this: callers that cannot call cudaMalloc, either because all of
// the device memory they may use was handed out up front to their own pool or
// arena (a long-running solver service that must not fail with out-of-memory
// in the middle of a request), or because they run on a latency-critical path
// where cudaMalloc/cudaFree would synchronise the device.  asyrk_residual needs
// a problem handle, whose creation allocates; this entry point needs nothing
// but the caller's arrays.
//
// Its only scratch (per-block partial sums and a completion counter) lives in
// the file-scope array g_noalloc_scratch below: a fixed 128 KiB + 64 B that
// every GPU which loads the library holds until the process exits.  Host code
// must not hand the array's name to a kernel (on the host it is only a
// stand-in); the device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, on the first call made on it.
#include <mutex>

#include "common.cuh"

#define NOALLOC_ROWS_PER_BLOCK 2048
#define NOALLOC_MAX_BLOCKS 8192
#define NOALLOC_MAX_DEVICES 64

namespace asyrk {

// [0, MAX_BLOCKS): partial sums of (b_i - a_i^T x)^2; [MAX_BLOCKS, 2 MAX_BLOCKS):
// partial sums of b_i^2; then one 8-byte completion counter (8 doubles of room).
static __device__ __align__(256) double g_noalloc_scratch[2 * NOALLOC_MAX_BLOCKS + 8];

__device__ __forceinline__ double noalloc_value(const double *v, int64_t k) { return v[k]; }
__device__ __forceinline__ double noalloc_value(const float *v, int64_t k) { return (double)v[k]; }
__device__ __forceinline__ double noalloc_value(const bf16_t *v, int64_t k)
{
    return (double)__uint_as_float(((unsigned)v[k].bits) << 16);
}

// One block per NOALLOC_ROWS_PER_BLOCK rows, 8 lanes per row.  Entries outside
// [0, nnz) or columns outside [0, n) are not read; they turn the result into NaN.
template <typename VT>
__global__ void __launch_bounds__(256)
k_residual_noalloc(int64_t m, int64_t n, int64_t nnz, const int64_t *__restrict__ row_ptr,
                   const int32_t *__restrict__ col, const VT *__restrict__ val,
                   const double *__restrict__ b, const double *__restrict__ x, double *scratch,
                   double *out)
{
    constexpr int G = 8;
    __shared__ double sh[2][8];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, sl = lane % G;
    const int grp = threadIdx.x / G;  // 32 row groups per block
    const int64_t row0 = (int64_t)blockIdx.x * NOALLOC_ROWS_PER_BLOCK;
    double rr = 0.0, bb = 0.0;
    bool bad = false;
    for (int it = 0; it < NOALLOC_ROWS_PER_BLOCK / 32; ++it) {
        const int64_t i = row0 + (int64_t)it * 32 + grp;
        double acc = 0.0;
        if (i < m) {
            int64_t s = row_ptr[i], e = row_ptr[i + 1];
            if (s < 0 || e > nnz || e < s) {
                bad = true;
                s = e = 0;
            }
            for (int64_t k = s + sl; k < e; k += G) {
                const int32_t c = col[k];
                if (c < 0 || (int64_t)c >= n) {
                    bad = true;
                    continue;
                }
                acc += noalloc_value(val, k) * x[c];
            }
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (i < m && sl == 0) {
            const double ri = b[i] - acc;
            rr += ri * ri;
            bb += b[i] * b[i];
        }
    }
    if (__any_sync(0xffffffffu, bad)) rr = __longlong_as_double(0x7ff8000000000000LL);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        rr += __shfl_xor_sync(0xffffffffu, rr, o);
        bb += __shfl_xor_sync(0xffffffffu, bb, o);
    }
    if (lane == 0) {
        sh[0][wid] = rr;
        sh[1][wid] = bb;
    }
    __syncthreads();
    unsigned long long *count =
        reinterpret_cast<unsigned long long *>(scratch + 2 * NOALLOC_MAX_BLOCKS);
    if (threadIdx.x == 0) {
        double a = 0.0, c = 0.0;
        for (int w = 0; w < 8; ++w) {
            a += sh[0][w];
            c += sh[1][w];
        }
        scratch[blockIdx.x] = a;
        scratch[NOALLOC_MAX_BLOCKS + blockIdx.x] = c;
        __threadfence();
        last = (atomicAdd(count, 1ull) == (unsigned long long)gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double a = 0.0, c = 0.0;
    for (unsigned k = threadIdx.x; k < gridDim.x; k += 256) {
        a += __ldcg(scratch + k);
        c += __ldcg(scratch + NOALLOC_MAX_BLOCKS + k);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if (lane == 0) {
        sh[0][wid] = a;
        sh[1][wid] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tc = 0.0;
        for (int w = 0; w < 8; ++w) {
            ta += sh[0][w];
            tc += sh[1][w];
        }
        out[0] = sqrt(ta);
        out[1] = sqrt(tc);
        *count = 0ull;  // the next call finds the counter at zero
    }
}

static std::mutex g_noalloc_mutex;
static double *g_noalloc_ptr[NOALLOC_MAX_DEVICES];

// Device address of the scratch array on the current device, looked up once
// per device (the first call on a device does this; it should come before any
// stream capture on that device).
static int noalloc_scratch(double **ptr)
{
    int dev = -1;
    ASYRK_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES)
        return set_error(ASYRK_EINVAL, "device ordinal %d is beyond %d", dev, NOALLOC_MAX_DEVICES);
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress", __FILE__, __LINE__);
        g_noalloc_ptr[dev] = static_cast<double *>(p);
    }
    *ptr = g_noalloc_ptr[dev];
    return ASYRK_OK;
}

}  // namespace asyrk

using namespace asyrk;

extern "C" int asyrk_residual_noalloc(int64_t m, int64_t n, int64_t nnz, const int64_t *row_ptr,
                                      const int32_t *col_idx, const void *values, int vdtype,
                                      const double *b, const double *x, double *out, void *stream)
{
    if (m < 1 || n < 1 || n > 0x7fffffffLL || nnz < 0)
        return set_error(ASYRK_EINVAL, "m and n must be >= 1 (n <= 2^31-1) and nnz >= 0");
    if (m > ASYRK_NOALLOC_MAX_ROWS)
        return set_error(ASYRK_EINVAL,
                         "m = %lld exceeds the %d rows the static scratch of "
                         "asyrk_residual_noalloc can hold",
                         (long long)m, ASYRK_NOALLOC_MAX_ROWS);
    if (!row_ptr || !col_idx || !values || !b || !x || !out)
        return set_error(ASYRK_EINVAL, "NULL array");
    if (vdtype != ASYRK_F64 && vdtype != ASYRK_F32 && vdtype != ASYRK_BF16)
        return set_error(ASYRK_EINVAL, "unknown value dtype %d", vdtype);
    double *scratch = nullptr;
    int st = noalloc_scratch(&scratch);
    if (st != ASYRK_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    // the completion counter must start at zero (a call cut short may have left it set)
    ASYRK_CK(cudaMemsetAsync(scratch + 2 * NOALLOC_MAX_BLOCKS, 0, sizeof(unsigned long long), s));
    const unsigned grid = (unsigned)((m + NOALLOC_ROWS_PER_BLOCK - 1) / NOALLOC_ROWS_PER_BLOCK);
    switch (vdtype) {
    case ASYRK_F64:
        k_residual_noalloc<double><<<grid, 256, 0, s>>>(m, n, nnz, row_ptr, col_idx,
                                                        (const double *)values, b, x, scratch, out);
        break;
    case ASYRK_F32:
        k_residual_noalloc<float><<<grid, 256, 0, s>>>(m, n, nnz, row_ptr, col_idx,
                                                       (const float *)values, b, x, scratch, out);
        break;
    default:
        k_residual_noalloc<bf16_t><<<grid, 256, 0, s>>>(m, n, nnz, row_ptr, col_idx,
                                                        (const bf16_t *)values, b, x, scratch, out);
        break;
    }
    ASYRK_CK(cudaGetLastError());
    return ASYRK_OK;
}
