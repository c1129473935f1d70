// measure.cu -- FP64 error measures and small vector kernels.
//
// The convergence check of a solve is ||x - x*|| / ||x*|| (with x* given) or
// ||b - A x|| / ||b|| (Section 5 plots ||Ax - b||), both accumulated in FP64
// on the GPU.  Reductions are deterministic: a fixed grid writes one partial
// per block and the last block to finish sums the partials in block order.
// The residual kernel also serves the refinement loop: r = b - A x64 in FP64,
// optionally stored (rounded to FP32) as the right-hand side of the inner solve.
#include "common.cuh"
#include "devmem.cuh"

namespace asyrk {

constexpr int RT = 256;  // threads per reduction block

template <int NV>
__device__ __forceinline__ void block_finish(double (&v)[NV], double *part, unsigned *count,
                                             double *out)
{
    __shared__ double sh[RT / 32][NV];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double t = v[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) sh[wid][q] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double t = 0.0;
            for (int w = 0; w < RT / 32; ++w) t += sh[w][q];
            part[q * ASYRK_MAX_RED_BLOCKS + blockIdx.x] = t;
        }
        __threadfence();
        last = (atomicAdd(count, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double t = 0.0;
        for (unsigned b = threadIdx.x; b < gridDim.x; b += RT)
            t += __ldcg(part + q * ASYRK_MAX_RED_BLOCKS + b);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) sh[wid][q] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double t = 0.0;
            for (int w = 0; w < RT / 32; ++w) t += sh[w][q];
            out[q] = t;
        }
        *count = 0u;
    }
}

static unsigned red_grid(int64_t work, int sm_count)
{
    int64_t g = (work + RT - 1) / RT;
    const int64_t cap = (int64_t)sm_count * 4 < ASYRK_MAX_RED_BLOCKS ? (int64_t)sm_count * 4
                                                                     : ASYRK_MAX_RED_BLOCKS;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (unsigned)g;
}

__device__ __forceinline__ double widen_x(const float *x, int64_t i) { return (double)x[i]; }
__device__ __forceinline__ double widen_x(const double *x, int64_t i) { return x[i]; }

template <typename XT>
__global__ void __launch_bounds__(RT) k_err2(const XT *__restrict__ x, const double *__restrict__ xt,
                                             int64_t n, double *part, unsigned *count, double *out)
{
    double v[2] = {0.0, 0.0};
    for (int64_t i = (int64_t)blockIdx.x * RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) {
        const double d = widen_x(x, i) - xt[i];
        v[0] += d * d;
        v[1] += xt[i] * xt[i];
    }
    block_finish<2>(v, part, count, out);
}

__global__ void __launch_bounds__(RT) k_sumsq(const double *__restrict__ a, int64_t n, double *part,
                                              unsigned *count, double *out)
{
    double v[1] = {0.0};
    for (int64_t i = (int64_t)blockIdx.x * RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT)
        v[0] += a[i] * a[i];
    block_finish<1>(v, part, count, out);
}

__device__ __forceinline__ double widen_v(const double *v, int64_t k) { return v[k]; }
__device__ __forceinline__ double widen_v(const float *v, int64_t k) { return (double)v[k]; }
__device__ __forceinline__ double widen_v(const bf16_t *v, int64_t k)
{
    return (double)__uint_as_float(((unsigned)v[k].bits) << 16);
}

// r_i = b_i - a_i^T x in FP64; 8 lanes per row, rows grid-strided.
template <typename VT, typename XT>
__global__ void __launch_bounds__(RT) k_residual(const RowRec *rec,
                                                 RowRec *rec_out, const int32_t *__restrict__ col,
                                                 const VT *__restrict__ val,
                                                 const double *__restrict__ b64,
                                                 const XT *__restrict__ x, int64_t m, double *part,
                                                 unsigned *count, double *out)
{
    constexpr int G = 8;
    const int lane = threadIdx.x & 31, sl = lane % G;
    const int64_t grp = ((int64_t)blockIdx.x * RT + threadIdx.x) / G;
    const int64_t ngrp = (int64_t)gridDim.x * RT / G;
    double v[1] = {0.0};
    const int64_t iters = (m + ngrp - 1) / ngrp;  // uniform trip count for the shuffles
    for (int64_t it = 0; it < iters; ++it) {
        const int64_t i = grp + it * ngrp;
        double acc = 0.0;
        if (i < m) {
            const RowRec r = rec[i];
            for (int64_t k = sl; k < (int64_t)r.len; k += G)
                acc += widen_v(val, r.start + k) * widen_x(x, col[r.start + k]);
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (i < m && sl == 0) {
            const double ri = b64[i] - acc;
            v[0] += ri * ri;
            if (rec_out) rec_out[i].b = (float)ri;
        }
    }
    block_finish<1>(v, part, count, out);
}

// g += A^T (A x - b), FP64: 8 lanes per row form r_i = a_i^T x - b_i, then each
// lane adds r_i * A_it into g_t with an FP64 atomic (the measure of Table 2 is
// ||g||^2).
template <typename VT, typename XT>
__global__ void __launch_bounds__(RT) k_normal_scatter(const RowRec *__restrict__ rec,
                                                       const int32_t *__restrict__ col,
                                                       const VT *__restrict__ val,
                                                       const double *__restrict__ b64,
                                                       const XT *__restrict__ x, int64_t m,
                                                       double *g)
{
    constexpr int G = 8;
    const int lane = threadIdx.x & 31, sl = lane % G;
    const int64_t grp = ((int64_t)blockIdx.x * RT + threadIdx.x) / G;
    const int64_t ngrp = (int64_t)gridDim.x * RT / G;
    const int64_t iters = (m + ngrp - 1) / ngrp;  // uniform trip count for the shuffles
    for (int64_t it = 0; it < iters; ++it) {
        const int64_t i = grp + it * ngrp;
        double acc = 0.0;
        RowRec r;
        r.len = 0;
        r.start = 0;
        if (i < m) {
            r = rec[i];
            for (int64_t k = sl; k < (int64_t)r.len; k += G)
                acc += widen_v(val, r.start + k) * widen_x(x, col[r.start + k]);
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (i < m) {
            const double ri = acc - b64[i];
            for (int64_t k = sl; k < (int64_t)r.len; k += G)
                atomicAdd(g + col[r.start + k], widen_v(val, r.start + k) * ri);
        }
    }
}

__global__ void k_convert_f64_f32(const double *__restrict__ s, float *__restrict__ d, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        d[i] = (float)s[i];
}

__global__ void k_convert_f32_f64(const float *__restrict__ s, double *__restrict__ d, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        d[i] = (double)s[i];
}

__global__ void k_axpy_f32_f64(double *__restrict__ x, const float *__restrict__ d, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] += (double)d[i];
}

__global__ void k_restore_b(RowRec *rec, const double *__restrict__ b64, int64_t m)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        rec[i].b = (float)b64[i];
}

static unsigned ew_grid(int64_t n)
{
    int64_t g = (n + 255) / 256;
    if (g > 4096) g = 4096;
    if (g < 1) g = 1;
    return (unsigned)g;
}

int launch_err2(asyrk_problem *p, const void *x, bool x_f64, const double *xt, int slot,
                cudaStream_t s)
{
    const unsigned g = red_grid(p->n, p->sm_count);
    if (x_f64)
        k_err2<double><<<g, RT, 0, s>>>((const double *)x, xt, p->n, p->red_part, p->red_count,
                                        p->red_out + slot);
    else
        k_err2<float><<<g, RT, 0, s>>>((const float *)x, xt, p->n, p->red_part, p->red_count,
                                       p->red_out + slot);
    ASYRK_CK(cudaGetLastError());
    p->launches += 1;
    return ASYRK_OK;
}

int launch_sumsq(asyrk_problem *p, const double *v, int64_t n, int slot, cudaStream_t s)
{
    const unsigned g = red_grid(n, p->sm_count);
    k_sumsq<<<g, RT, 0, s>>>(v, n, p->red_part, p->red_count, p->red_out + slot);
    ASYRK_CK(cudaGetLastError());
    p->launches += 1;
    return ASYRK_OK;
}

template <typename VT>
static void residual_vt(asyrk_problem *p, const void *x, bool x_f64, RowRec *rec_out,
                        unsigned g, int slot, cudaStream_t s)
{
    const VT *val = (const VT *)p->val;
    if (x_f64)
        k_residual<VT, double><<<g, RT, 0, s>>>(p->rec, rec_out, p->col, val, p->b64,
                                                (const double *)x, p->m, p->red_part,
                                                p->red_count, p->red_out + slot);
    else
        k_residual<VT, float><<<g, RT, 0, s>>>(p->rec, rec_out, p->col, val, p->b64,
                                               (const float *)x, p->m, p->red_part, p->red_count,
                                               p->red_out + slot);
}

int launch_residual(asyrk_problem *p, const void *x, bool x_f64, bool write_rec_b, int slot,
                    cudaStream_t s)
{
    const unsigned g = red_grid(p->m * 8, p->sm_count);
    RowRec *ro = write_rec_b ? p->rec : nullptr;
    switch (p->dtype) {
    case ASYRK_F64: residual_vt<double>(p, x, x_f64, ro, g, slot, s); break;
    case ASYRK_F32: residual_vt<float>(p, x, x_f64, ro, g, slot, s); break;
    default: residual_vt<bf16_t>(p, x, x_f64, ro, g, slot, s); break;
    }
    ASYRK_CK(cudaGetLastError());
    p->launches += 1;
    if (write_rec_b) p->rec_b_is_residual = true;
    return ASYRK_OK;
}

template <typename VT>
static void normal_vt(asyrk_problem *p, const void *x, bool x_f64, unsigned g, cudaStream_t s)
{
    const VT *val = (const VT *)p->val;
    if (x_f64)
        k_normal_scatter<VT, double><<<g, RT, 0, s>>>(p->rec, p->col, val, p->b64,
                                                      (const double *)x, p->m, p->g64);
    else
        k_normal_scatter<VT, float><<<g, RT, 0, s>>>(p->rec, p->col, val, p->b64,
                                                     (const float *)x, p->m, p->g64);
}

int launch_normal_residual(asyrk_problem *p, const void *x, bool x_f64, int slot, cudaStream_t s)
{
    if (!p->g64) {
        const int st = devmem_alloc_n(&p->g64, (size_t)p->n, s);  // ordered on s, used on s
        if (st != ASYRK_OK) return st;
        p->dev_bytes += p->n * (int64_t)sizeof(double);
    }
    ASYRK_CK(cudaMemsetAsync(p->g64, 0, p->n * sizeof(double), s));
    int64_t g = (p->m * 8 + RT - 1) / RT;
    const int64_t cap = (int64_t)p->sm_count * 8;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    switch (p->dtype) {
    case ASYRK_F64: normal_vt<double>(p, x, x_f64, (unsigned)g, s); break;
    case ASYRK_F32: normal_vt<float>(p, x, x_f64, (unsigned)g, s); break;
    default: normal_vt<bf16_t>(p, x, x_f64, (unsigned)g, s); break;
    }
    ASYRK_CK(cudaGetLastError());
    p->launches += 1;
    return launch_sumsq(p, p->g64, p->n, slot, s);
}

int launch_convert(const void *src, bool src_f64, void *dst, bool dst_f64, int64_t n,
                   cudaStream_t s)
{
    if (src_f64 == dst_f64) {
        ASYRK_CK(cudaMemcpyAsync(dst, src, n * (src_f64 ? 8 : 4), cudaMemcpyDeviceToDevice, s));
        return ASYRK_OK;
    }
    if (src_f64)
        k_convert_f64_f32<<<ew_grid(n), 256, 0, s>>>((const double *)src, (float *)dst, n);
    else
        k_convert_f32_f64<<<ew_grid(n), 256, 0, s>>>((const float *)src, (double *)dst, n);
    ASYRK_CK(cudaGetLastError());
    return ASYRK_OK;
}

int launch_axpy_f32_to_f64(double *x64, const float *d, int64_t n, cudaStream_t s)
{
    k_axpy_f32_f64<<<ew_grid(n), 256, 0, s>>>(x64, d, n);
    ASYRK_CK(cudaGetLastError());
    return ASYRK_OK;
}

int launch_restore_rec_b(asyrk_problem *p, cudaStream_t s)
{
    k_restore_b<<<ew_grid(p->m), 256, 0, s>>>(p->rec, p->b64, p->m);
    ASYRK_CK(cudaGetLastError());
    p->launches += 1;
    p->rec_b_is_residual = false;
    return ASYRK_OK;
}

}  // namespace asyrk
