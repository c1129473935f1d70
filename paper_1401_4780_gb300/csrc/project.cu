// project.cu -- the row-projection kernels (the method's hot loop).
//
// Worker w applies projections t = w, w + W, w + 2W, ... of the launch
// (W = number of workers), projection t being number j = j0 + t of the
// problem's row sequence; the per-projection steps are in worker.cuh.
//
// With sequential = true a single worker (one warp) applies the projections
// strictly in order, fencing its updates before the next gather: the
// sequential RK iterate of Eq. (2).
#include "worker.cuh"

namespace asyrk {

// 5 blocks of 256 per SM (<= 48 registers) with an FP32 iterate and G > 1; 4
// (<= 64) with FP64 values in flight or one lane walking a whole row
template <typename VT, typename XT, int G, bool SEQ, bool EXCL>
__global__ void __launch_bounds__(256, (sizeof(XT) == 4 && G > 1 ? 5 : 4)) k_project(const ProjArgs a)
{
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned long long skipped = run_workers<VT, XT, G, SEQ, EXCL>(a, warp * (32 / G),
                                                                         a.workers);
    if (EXCL && skipped) atomicAdd(a.skipped, skipped);
}

__global__ void k_draw_rows(const RowRec *__restrict__ rec, uint2 key, unsigned m, int uniform,
                            unsigned stream_id, unsigned long long j0, long long count,
                            int sampling, int shuf_h, int32_t *__restrict__ out)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    const unsigned long long j = j0 + (unsigned long long)t;
    if (sampling == 1) {
        out[t] = (int32_t)shuffled_position(j, m, stream_id, key, shuf_h);
    } else {
        RowRec r;
        out[t] = (int32_t)draw_row(j, stream_id, key, m, uniform, rec, r);
    }
}

// ---------------------------------------------------------------------------
// dispatch
// ---------------------------------------------------------------------------
using KernelFn = ProjKernelFn;

// launches with at most this many warps per SM run the latency form (project_pf.cu)
constexpr long long LATENCY_FORM_WARPS_PER_SM = 8;

template <typename VT, typename XT, bool SEQ, bool EXCL>
static KernelFn pick_g(int G)
{
    switch (G) {
    case 1: return k_project<VT, XT, 1, SEQ, EXCL>;
    case 2: return k_project<VT, XT, 2, SEQ, EXCL>;
    case 4: return k_project<VT, XT, 4, SEQ, EXCL>;
    case 8: return k_project<VT, XT, 8, SEQ, EXCL>;
    case 16: return k_project<VT, XT, 16, SEQ, EXCL>;
    case 32: return k_project<VT, XT, 32, SEQ, EXCL>;
    default: return nullptr;
    }
}

template <typename VT>
static KernelFn pick_x(bool x_f64, bool seq, bool excl, int G)
{
    if (seq) return x_f64 ? pick_g<VT, double, true, false>(G) : nullptr;
    if (excl)
        return x_f64 ? pick_g<VT, double, false, true>(G) : pick_g<VT, float, false, true>(G);
    return x_f64 ? pick_g<VT, double, false, false>(G) : pick_g<VT, float, false, false>(G);
}

static KernelFn pick_kernel(int dtype, bool x_f64, bool seq, bool excl, int G)
{
    switch (dtype) {
    case ASYRK_F64: return pick_x<double>(x_f64, seq, excl, G);
    case ASYRK_F32: return pick_x<float>(x_f64, seq, excl, G);
    case ASYRK_BF16: return pick_x<bf16_t>(x_f64, seq, excl, G);
    default: return nullptr;
    }
}

int choose_subwarp(int64_t max_len, int64_t nnz, int64_t m)
{
    // one 4-entry chunk per lane for the longest rows, capped at a full warp
    (void)nnz;
    (void)m;
    int G = 2;
    while (G < 32 && 4 * G < max_len) G *= 2;
    return G;
}

int project_max_workers(const asyrk_problem *p, bool x_f64, int subwarp, int *max_workers)
{
    KernelFn k = pick_kernel(p->dtype, x_f64, false, true, subwarp);
    if (!k) return set_error(ASYRK_EINVAL, "no projection kernel for subwarp %d", subwarp);
    int per_sm = 0;
    ASYRK_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, 0));
    if (per_sm < 1) per_sm = 1;
    *max_workers = per_sm * p->sm_count * (256 / subwarp);
    return ASYRK_OK;
}

int launch_project(const ProjectLaunch &L)
{
    asyrk_problem *p = L.p;
    if (L.count == 0) return ASYRK_OK;
    const bool excl = L.exclusive && !L.sequential;
    KernelFn k = nullptr;
    const bool few_warps =
        ((long long)L.workers * L.subwarp + 31) / 32 <= LATENCY_FORM_WARPS_PER_SM * p->sm_count;
    if (!L.sequential && L.update == 0 && (L.form > 0 || (L.form == 0 && few_warps)))
        k = pick_project_pf(p->dtype, L.x_f64, excl, L.subwarp);
    if (!k) k = pick_kernel(p->dtype, L.x_f64, L.sequential, excl, L.subwarp);
    if (!k) return set_error(ASYRK_EINVAL, "no projection kernel for subwarp %d", L.subwarp);
    ProjArgs a;
    a.rec = p->rec;
    a.col = p->col;
    a.val = p->val;
    a.x = L.x;
    a.b64 = p->b64;
    a.w64 = p->w64;
    a.key = make_uint2((unsigned)p->seed, (unsigned)(p->seed >> 32));
    a.m = (unsigned)p->m;
    a.uniform = p->uniform;
    a.stream_id = L.stream_id;
    a.j0 = L.j0;
    a.count = L.count;
    a.gamma = L.gamma;
    a.bvec = nullptr;
    a.sampling = L.sampling;
    a.shuf_h = shuffle_half_bits(p->m);
    a.update = L.update;
    a.busy = p->busy;
    a.skipped = p->skipped;
    a.dyn = L.dyn;
    if (L.sequential) {
        a.workers = 1;
        k<<<1, 32, 0, L.stream>>>(a);
    } else {
        a.workers = L.workers;
        const long long threads = (long long)L.workers * L.subwarp;
        const long long blocks = (threads + 255) / 256;
        k<<<(unsigned)blocks, 256, 0, L.stream>>>(a);
    }
    ASYRK_CK(cudaGetLastError());
    p->launches += 1;
    return ASYRK_OK;
}

int launch_draw_rows(const asyrk_problem *p, unsigned long long j0, int64_t count,
                     unsigned stream_id, int sampling, int32_t *rows_dev, cudaStream_t s)
{
    const uint2 key = make_uint2((unsigned)p->seed, (unsigned)(p->seed >> 32));
    const long long blocks = (count + 255) / 256;
    k_draw_rows<<<(unsigned)blocks, 256, 0, s>>>(p->rec, key, (unsigned)p->m, p->uniform,
                                                   stream_id, j0, count, sampling,
                                                   shuffle_half_bits(p->m), rows_dev);
    ASYRK_CK(cudaGetLastError());
    return ASYRK_OK;
}

}  // namespace asyrk
