// project_pf.cu -- the latency form of the row-projection kernel (worker.cuh,
// run_workers_pf): for launches with a few warps per SM, where a worker's
// projections would otherwise wait on their row record, row and gathers one
// after another.  Same projections, order per worker and delay as k_project.
#include "worker.cuh"

namespace asyrk {

// few warps per SM by construction: the registers that hold a worker's next
// projections are not short
template <typename VT, typename XT, int G, bool EXCL>
__global__ void __launch_bounds__(256, 2) k_project_pf(const ProjArgs a)
{
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned long long skipped = run_workers_pf<VT, XT, G, EXCL>(a, warp * (32 / G),
                                                                       a.workers);
    if (EXCL && skipped) atomicAdd(a.skipped, skipped);
}

template <typename VT, typename XT, bool EXCL>
static ProjKernelFn pick_pf_g(int G)
{
    switch (G) {
    case 1: return k_project_pf<VT, XT, 1, EXCL>;
    case 2: return k_project_pf<VT, XT, 2, EXCL>;
    case 4: return k_project_pf<VT, XT, 4, EXCL>;
    case 8: return k_project_pf<VT, XT, 8, EXCL>;
    case 16: return k_project_pf<VT, XT, 16, EXCL>;
    case 32: return k_project_pf<VT, XT, 32, EXCL>;
    default: return nullptr;
    }
}

template <typename VT>
static ProjKernelFn pick_pf_x(bool x_f64, bool excl, int G)
{
    if (excl) return x_f64 ? pick_pf_g<VT, double, true>(G) : pick_pf_g<VT, float, true>(G);
    return x_f64 ? pick_pf_g<VT, double, false>(G) : pick_pf_g<VT, float, false>(G);
}

ProjKernelFn pick_project_pf(int dtype, bool x_f64, bool excl, int G)
{
    switch (dtype) {
    case ASYRK_F64: return pick_pf_x<double>(x_f64, excl, G);
    case ASYRK_F32: return pick_pf_x<float>(x_f64, excl, G);
    case ASYRK_BF16: return pick_pf_x<bf16_t>(x_f64, excl, G);
    default: return nullptr;
    }
}

}  // namespace asyrk
