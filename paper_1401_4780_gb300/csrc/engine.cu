// engine.cu -- kernels of the multi-system engine (see batch.cuh).
#include <math.h>

#include "batch.cuh"
#include "worker.cuh"

namespace asyrk {

// Cor. 2 asks 2 e lambda_max (tau + 1) / m <= 1 for near-linear speedup.  With
// no lambda_max at hand the estimate uses Section 1's value for row-normalised
// Gaussian matrices, lambda_max ~ (1 + sqrt(m/n))^2.
long long tau_cap_estimate(int64_t m, int64_t n)
{
    const double ratio = (double)m / (double)n;
    const double lmax = (1.0 + sqrt(ratio)) * (1.0 + sqrt(ratio));
    const double cap = (double)m / (2.0 * M_E * lmax) - 1.0;
    return cap < 1.0 ? 1LL : (long long)cap;
}

// ---------------------------------------------------------------------------
// plan: one block; each thread owns slots tid, tid + blockDim, ...
// ---------------------------------------------------------------------------
constexpr int PLAN_THREADS = 1024;
constexpr int PLAN_PER_THREAD = BATCH_MAX_SLOTS / PLAN_THREADS;

template <typename T, typename Op>
__device__ __forceinline__ T block_all(T v, Op op, T *sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    T r = sh[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = op(r, sh[w]);
    __syncthreads();
    return r;
}

// exclusive prefix sum over the block; *total receives the block's sum
__device__ __forceinline__ long long block_excl_scan(long long v, long long *sh, long long &total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    __syncthreads();
    if (lane == 31) sh[wid] = incl;
    __syncthreads();
    long long before = 0, tot = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
        if (k < wid) before += sh[k];
        tot += sh[k];
    }
    __syncthreads();
    total = tot;
    return before + incl - v;
}

__global__ void __launch_bounds__(PLAN_THREADS) k_batch_plan(SysDesc *d, int count, int R,
                                                              int even_share)
{
    __shared__ double shd[32];
    __shared__ long long shl[32];
    const int tid = threadIdx.x;
    auto add_d = [](double a, double b) { return a + b; };
    auto max_d = [](double a, double b) { return a > b ? a : b; };
    auto add_l = [](long long a, long long b) { return a + b; };
    double work[PLAN_PER_THREAD], chain[PLAN_PER_THREAD];
    int cap[PLAN_PER_THREAD], w[PLAN_PER_THREAD];
    bool on[PLAN_PER_THREAD];
    double wt = 0.0;
    long long na = 0;
#pragma unroll
    for (int q = 0; q < PLAN_PER_THREAD; ++q) {
        const int s = tid + q * PLAN_THREADS;
        on[q] = s < count && d[s].active && d[s].phase == 0;
        work[q] = on[q] ? d[s].work : 0.0;
        cap[q] = on[q] ? (d[s].cap_warps > 0 ? d[s].cap_warps : 1) : 0;
        // projections per worker per sweep with one warp (32/G workers)
        chain[q] = on[q] ? (double)d[s].m / (double)(32 / (d[s].G > 0 ? d[s].G : 32)) : 0.0;
        wt += work[q];
        na += on[q] ? 1 : 0;
    }
    const double wtot = block_all(wt, add_d, shd);
    const long long nact = block_all(na, add_l, shl);
    // with even_share, half of the warps evenly (short, latency-bound solves get
    // parallelism); the rest in proportion to the work per sweep.  Every active
    // slot gets at least one warp and at most its cap; the total stays <= R.
    long long even = nact > 0 ? 1 : 0;
    if (even_share && nact > 0 && R / (2 * nact) > 1) even = R / (2 * nact);
    long long u = 0;
#pragma unroll
    for (int q = 0; q < PLAN_PER_THREAD; ++q) {
        w[q] = on[q] ? (int)(even < cap[q] ? even : cap[q]) : 0;
        u += w[q];
    }
    long long used = block_all(u, add_l, shl);
    for (int pass = 0; pass < 2 && used < R && wtot > 0.0; ++pass) {
        double wu = 0.0;
#pragma unroll
        for (int q = 0; q < PLAN_PER_THREAD; ++q)
            if (on[q] && w[q] < cap[q]) wu += work[q];
        const double wunc = block_all(wu, add_d, shd);
        if (wunc <= 0.0) break;
        const long long left = R - used;
        long long a_sum = 0;
#pragma unroll
        for (int q = 0; q < PLAN_PER_THREAD; ++q) {
            if (!on[q] || w[q] >= cap[q]) continue;
            long long a = (long long)((double)left * work[q] / wunc);
            if (a > cap[q] - w[q]) a = cap[q] - w[q];
            w[q] += (int)a;
            a_sum += a;
        }
        used += block_all(a_sum, add_l, shl);
    }
    // sweeps this step: each slot's worker chain (projections per worker for
    // its k sweeps) should not outlast the longest single-sweep chain
    double tl = 0.0;
#pragma unroll
    for (int q = 0; q < PLAN_PER_THREAD; ++q)
        if (on[q] && w[q] > 0 && chain[q] / w[q] > tl) tl = chain[q] / w[q];
    double tmax = block_all(tl, max_d, shd);
    // the server's step runs at least SERVER_STEP_CHAIN projections per worker,
    // so that a lone request whose sweep is short does several sweeps per step
    // and pays the step's fixed cost (plan, check, the host's round trip) less
    // often; it checks its tolerance once per step
    if (even_share && tmax < SERVER_STEP_CHAIN) tmax = SERVER_STEP_CHAIN;
    // warp ranges: exclusive prefix of the warps in slot order, one stride row
    // (slots q*PLAN_THREADS .. q*PLAN_THREADS + PLAN_THREADS - 1) at a time
    long long base = 0;
#pragma unroll
    for (int q = 0; q < PLAN_PER_THREAD; ++q) {
        long long row_total = 0;
        const long long ex = block_excl_scan((long long)w[q], shl, row_total);
        const int s = tid + q * PLAN_THREADS;
        if (s < count) {
            long long w0 = base + ex, nw = w[q];
            if (w0 >= R) {
                w0 = R;
                nw = 0;
            } else if (w0 + nw > R) {
                nw = R - w0;
            }
            int kk = 1;
            if (on[q] && nw > 0 && tmax > 0.0) {
                const double kf = tmax / (chain[q] / (double)nw);
                long long kmax = d[s].max_k > 1 ? d[s].max_k : 1;
                const long long left_sw = d[s].max_sweeps - d[s].sweeps;
                if (kmax > left_sw) kmax = left_sw > 1 ? left_sw : 1;
                kk = kf >= (double)kmax ? (int)kmax : (kf < 1.0 ? 1 : (int)kf);
            }
            if (even_share && on[q] && kk > 1) {
                // server steps: no more sweeps than the slot still needs at the
                // contraction per sweep it has shown (its measure over its first,
                // or for an inner solve of refinement, over 1 at d = 0)
                const SysDesc &D = d[s];
                const bool inner = D.mode == SLOT_REFINE;
                const long long done = inner ? D.inner_sweeps : D.sweeps;
                const double m0 = inner ? 1.0 : D.meas0;
                const double target = inner ? D.inner_goal : D.tol;
                if (done > 0 && D.meas > 0.0 && m0 > 0.0 && D.meas < m0 && target > 0.0 &&
                    target < D.meas) {
                    const double rho = pow(D.meas / m0, 1.0 / (double)done);
                    const double rem = log(target / D.meas) / log(rho);
                    if (rem < (double)kk) kk = rem < 1.0 ? 1 : (int)ceil(rem);
                }
            }
            d[s].warp0 = (int)w0;
            d[s].nwarps = (int)nw;
            d[s].k = kk;
            if (d[s].first_nwarps == 0) d[s].first_nwarps = (int)nw;  // reported workers
        }
        base += row_total;
    }
}

// largest slot index whose start (warp0 or chunk0) is <= key
__device__ __forceinline__ int find_slot_warp(const SysDesc *d, int count, int key)
{
    int lo = 0, hi = count - 1, s = -1;
    while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        if (d[mid].warp0 <= key) {
            s = mid;
            lo = mid + 1;
        } else {
            hi = mid - 1;
        }
    }
    return s;
}

__device__ __forceinline__ int find_slot_chunk(const SysDesc *d, int count, int key)
{
    int lo = 0, hi = count - 1, s = -1;
    while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        if (d[mid].chunk0 <= key) {
            s = mid;
            lo = mid + 1;
        } else {
            hi = mid - 1;
        }
    }
    return s;
}

// ---------------------------------------------------------------------------
// project: one sweep of every active slot
// ---------------------------------------------------------------------------
template <typename VT, int G, bool EXCL>
__device__ __forceinline__ unsigned long long batch_run(const ProjArgs &a, int rel_warp)
{
    return run_workers<VT, float, G, false, EXCL, false>(a, (long long)rel_warp * (32 / G),
                                                         a.workers);
}

template <typename VT, bool EXCL>
__device__ __forceinline__ unsigned long long batch_run_g(const ProjArgs &a, int G, int rel_warp)
{
    switch (G) {
    case 1: return batch_run<VT, 1, EXCL>(a, rel_warp);
    case 2: return batch_run<VT, 2, EXCL>(a, rel_warp);
    case 4: return batch_run<VT, 4, EXCL>(a, rel_warp);
    case 8: return batch_run<VT, 8, EXCL>(a, rel_warp);
    case 16: return batch_run<VT, 16, EXCL>(a, rel_warp);
    default: return batch_run<VT, 32, EXCL>(a, rel_warp);
    }
}

template <bool EXCL>
__global__ void __launch_bounds__(256, 4) k_batch_project(SysDesc *d, int count)  // <= 64 registers
{
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int s = find_slot_warp(d, count, gw);
    if (s < 0) return;
    const SysDesc &D = d[s];
    if (!D.active || D.phase != 0 || gw >= D.warp0 + D.nwarps) return;  // warp-uniform
    // the warp's launch arguments live in shared memory, not registers
    __shared__ ProjArgs sa[8];
    ProjArgs &a = sa[threadIdx.x >> 5];
    if ((threadIdx.x & 31) == 0) {
        a.rec = D.rec;
        a.col = D.col;
        a.val = D.val;
        a.x = D.x;
        a.b64 = nullptr;
        a.w64 = nullptr;
        a.key = D.key;
        a.m = D.m;
        a.uniform = D.uniform;
        a.stream_id = D.stream_id;
        a.j0 = D.j;
        a.count = (unsigned long long)D.m * (unsigned long long)(D.k > 1 ? D.k : 1);  // k sweeps
        a.workers = (long long)D.nwarps * (32 / D.G);
        a.gamma = (double)D.gamma;
        a.bvec = D.bvec;
        a.sampling = D.sampling;
        a.shuf_h = D.shuf_h;
        a.update = D.update;
        a.busy = D.busy;
        a.skipped = nullptr;
        a.dyn = nullptr;
    }
    __syncwarp();
    const int rel = gw - D.warp0;
    const unsigned long long sk = (D.dtype == ASYRK_BF16)
                                      ? batch_run_g<bf16_t, EXCL>(a, D.G, rel)
                                      : batch_run_g<float, EXCL>(a, D.G, rel);
    if (EXCL && sk) atomicAdd(&d[s].skipped, sk);
}

// ---------------------------------------------------------------------------
// block reduction of two doubles; returns true in thread 0 of the last block
// of the slot to finish (which then holds the slot's totals in t0, t1)
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool slot_reduce(double v0, double v1, double *part, int chunk,
                                            int chunk0, int nchunks, unsigned *counter,
                                            double &t0, double &t1)
{
    __shared__ double sh[2][8];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v0 += __shfl_xor_sync(0xffffffffu, v0, o);
        v1 += __shfl_xor_sync(0xffffffffu, v1, o);
    }
    if (lane == 0) {
        sh[0][wid] = v0;
        sh[1][wid] = v1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < 8; ++w) {
            a += sh[0][w];
            b += sh[1][w];
        }
        part[2 * chunk] = a;
        part[2 * chunk + 1] = b;
        __threadfence();
        last = (atomicAdd(counter, 1u) == (unsigned)nchunks - 1u);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < nchunks; k += 256) {
        a += __ldcg(part + 2 * (chunk0 + k));
        b += __ldcg(part + 2 * (chunk0 + k) + 1);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    __syncthreads();
    if (lane == 0) {
        sh[0][wid] = a;
        sh[1][wid] = b;
    }
    __syncthreads();
    if (threadIdx.x != 0) return false;
    t0 = 0.0;
    t1 = 0.0;
    for (int w = 0; w < 8; ++w) {
        t0 += sh[0][w];
        t1 += sh[1][w];
    }
    *counter = 0u;
    return true;
}

__device__ __forceinline__ double slot_value(int dtype, const void *val, long long k)
{
    if (dtype == ASYRK_BF16)
        return (double)__uint_as_float(((unsigned)static_cast<const bf16_t *>(val)[k].bits) << 16);
    return (double)static_cast<const float *>(val)[k];
}

// measure_only: the first measure before any sweep (also ||x*|| when ref < 0)
__global__ void __launch_bounds__(256) k_batch_check(SysDesc *d, int count, double *part,
                                                     int measure_only)
{
    const int c = blockIdx.x;
    const int s = find_slot_chunk(d, count, c);
    if (s < 0) return;
    SysDesc &D = d[s];
    if (c >= D.chunk0 + D.nchunks) return;
    if (!D.active || (!measure_only && D.nwarps == 0)) return;  // same for all blocks of s
    const int k = c - D.chunk0;
    double v0 = 0.0, v1 = 0.0;
    if (D.xt && D.mode == SLOT_PLAIN) {
        const long long lo = (long long)k * BATCH_ERR_CHUNK;
        long long hi = lo + BATCH_ERR_CHUNK;
        if (hi > D.n) hi = D.n;
        for (long long t = lo + threadIdx.x; t < hi; t += 256) {
            const double e = (double)__ldcg(D.x + t) - D.xt[t];
            v0 += e * e;
            v1 += D.xt[t] * D.xt[t];
        }
    } else {
        const long long lo = (long long)k * BATCH_ROW_CHUNK;
        long long hi = lo + BATCH_ROW_CHUNK;
        if (hi > D.m) hi = D.m;
        for (long long i = lo + threadIdx.x; i < hi; i += 256) {
            const RowRec r = D.rec[i];
            double acc = 0.0;
            for (unsigned q = 0; q < r.len; ++q)
                acc += slot_value(D.dtype, D.val, r.start + q) *
                       (double)__ldcg(D.x + D.col[r.start + q]);
            const double bi = D.bvec ? (double)D.bvec[i] : (double)r.b;
            const double ri = bi - acc;
            v0 += ri * ri;
            v1 += bi * bi;
        }
    }
    double t0, t1;
    if (!slot_reduce(v0, v1, part, c, D.chunk0, D.nchunks, &D.chk_count, t0, t1)) return;
    if (D.ref < 0.0) D.ref = sqrt(t1) > 0.0 ? sqrt(t1) : 1.0;
    const double meas = sqrt(t0) / D.ref;
    D.meas = meas;
    if (measure_only) {
        D.meas0 = meas;
        if (meas <= D.tol) {
            D.active = 0;
            D.status = ASYRK_OK;
        } else if (D.max_sweeps <= 0) {
            D.active = 0;
            D.status = ASYRK_NOT_CONVERGED;
        }
        return;
    }
    const int ksw = D.k > 1 ? D.k : 1;
    D.j += (unsigned long long)D.m * (unsigned long long)ksw;
    D.sweeps += ksw;
    if (D.meas0 < 0.0) D.meas0 = meas;  // slots started without a first measure
    if (D.mode == SLOT_REFINE) {  // inner solve of A d = r: hand over to the outer step
        D.inner_sweeps += ksw;
        if (!isfinite(meas)) {
            D.active = 0;
            D.status = ASYRK_DIVERGED;
        } else if (meas <= D.inner_goal || D.inner_sweeps >= D.max_inner ||
                   D.sweeps >= D.max_sweeps) {
            D.phase = 1;
        }
        return;
    }
    if (!isfinite(meas) || meas > 1e30 * (D.meas0 > 0.0 ? D.meas0 : 1.0)) {
        D.active = 0;
        D.status = ASYRK_DIVERGED;
    } else if (meas <= D.tol) {
        D.active = 0;
        D.status = ASYRK_OK;
    } else if (D.sweeps >= D.max_sweeps) {
        D.active = 0;
        D.status = ASYRK_NOT_CONVERGED;
    }
}

// final ||b - A x64|| and ||b|| in FP64 per slot (row chunks)
__global__ void __launch_bounds__(256) k_batch_residual(SysDesc *d, int count, double *part)
{
    const int c = blockIdx.x;
    const int s = find_slot_chunk(d, count, c);
    if (s < 0) return;
    SysDesc &D = d[s];
    if (c >= D.chunk0 + D.nchunks) return;
    const int k = c - D.chunk0;
    double v0 = 0.0, v1 = 0.0;
    const long long lo = (long long)k * BATCH_ROW_CHUNK;
    long long hi = lo + BATCH_ROW_CHUNK;
    if (hi > D.m) hi = D.m;
    for (long long i = lo + threadIdx.x; i < hi; i += 256) {
        const RowRec r = D.rec[i];
        double acc = 0.0;
        for (unsigned q = 0; q < r.len; ++q)
            acc += slot_value(D.dtype, D.val, r.start + q) * D.x64[D.col[r.start + q]];
        const double ri = D.b64[i] - acc;
        v0 += ri * ri;
        v1 += D.b64[i] * D.b64[i];
    }
    double t0, t1;
    if (!slot_reduce(v0, v1, part, c, D.chunk0, D.nchunks, &D.res_count, t0, t1)) return;
    D.res2 = t0;
    D.bb2 = t1;
}

// outer step, part 1: x64 += d and d = 0 over the slot's x entries
__global__ void __launch_bounds__(256) k_batch_outer_update(SysDesc *d, int count)
{
    const int c = blockIdx.x;
    const int s = find_slot_chunk(d, count, c);
    if (s < 0) return;
    SysDesc &D = d[s];
    if (c >= D.chunk0 + D.nchunks || !D.active || D.mode != SLOT_REFINE || D.phase != 1) return;
    const long long lo = (long long)(c - D.chunk0) * BATCH_ERR_CHUNK;
    long long hi = lo + BATCH_ERR_CHUNK;
    if (hi > D.n) hi = D.n;
    for (long long t = lo + threadIdx.x; t < hi; t += 256) {
        D.x64[t] += (double)D.x[t];
        D.x[t] = 0.f;
    }
}

// outer step, part 2: r = b - A x64 (FP64) into r32, ||r||, ||x64 - x*||, decision
__global__ void __launch_bounds__(256) k_batch_outer_residual(SysDesc *d, int count, double *part)
{
    const int c = blockIdx.x;
    const int s = find_slot_chunk(d, count, c);
    if (s < 0) return;
    SysDesc &D = d[s];
    if (c >= D.chunk0 + D.nchunks || !D.active || D.mode != SLOT_REFINE || D.phase != 1) return;
    const int k = c - D.chunk0;
    double v0 = 0.0, v1 = 0.0;
    {
        const long long lo = (long long)k * BATCH_ROW_CHUNK;
        long long hi = lo + BATCH_ROW_CHUNK;
        if (hi > D.m) hi = D.m;
        for (long long i = lo + threadIdx.x; i < hi; i += 256) {
            const RowRec r = D.rec[i];
            double acc = 0.0;
            for (unsigned q = 0; q < r.len; ++q)
                acc += slot_value(D.dtype, D.val, r.start + q) * D.x64[D.col[r.start + q]];
            const double ri = D.b64[i] - acc;
            D.r32[i] = (float)ri;
            v0 += ri * ri;
        }
    }
    if (D.xt) {
        const long long lo = (long long)k * BATCH_ERR_CHUNK;
        long long hi = lo + BATCH_ERR_CHUNK;
        if (hi > D.n) hi = D.n;
        for (long long t = lo + threadIdx.x; t < hi; t += 256) {
            const double e = D.x64[t] - D.xt[t];
            v1 += e * e;
        }
    }
    double t0, t1;
    if (!slot_reduce(v0, v1, part, c, D.chunk0, D.nchunks, &D.out_count, t0, t1)) return;
    const double rnorm = sqrt(t0);
    // outer measure: ||x64 - x*|| / ||x*|| with x*, else ||b - A x64|| / ||b||
    const double meas = D.xt ? sqrt(t1) / D.outer_ref : rnorm / D.outer_ref;
    D.meas = meas;
    if (D.meas0 < 0.0) D.meas0 = meas;
    D.outer_steps += 1;
    D.res2 = t0;
    if (!isfinite(meas) || meas > 1e30 * (D.meas0 > 0.0 ? D.meas0 : 1.0)) {
        D.active = 0;
        D.status = ASYRK_DIVERGED;
    } else if (meas <= D.tol || rnorm == 0.0) {
        D.active = 0;
        D.status = ASYRK_OK;
    } else if (D.sweeps >= D.max_sweeps) {
        D.active = 0;
        D.status = ASYRK_NOT_CONVERGED;
    } else {
        D.phase = 0;  // next inner solve of A d = r
        D.ref = rnorm;
        D.inner_sweeps = 0;
        D.inner_goal = refine_inner_goal(D.inner_tol, D.tol, meas);
    }
}

// d_iter[0]: iterations done, d_iter[1]: the iteration bound
__global__ void k_batch_cond(SysDesc *d, int count, int *d_active, int *d_iter, int use_cond,
                             cudaGraphConditionalHandle h)
{
    __shared__ int sh[8];
    int a = 0;
    for (int s = threadIdx.x; s < count; s += blockDim.x) a += d[s].active;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += sh[w];
        *d_active = tot;
        const int it = d_iter[0] + 1;
        d_iter[0] = it;
        if (use_cond) cudaGraphSetConditional(h, (tot > 0 && it < d_iter[1]) ? 1u : 0u);
    }
}

__global__ void k_batch_convert(const double *x64, float *x, int64_t n, int to_f32, double *out64,
                                const float *in32)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (to_f32)
            x[i] = (float)x64[i];
        else
            out64[i] = (double)in32[i];
    }
}

int batch_resident_warps(int sm_count, bool excl, int *warps)
{
    int per_sm = 0;
    if (excl)
        ASYRK_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_project<true>, 256, 0));
    else
        ASYRK_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_project<false>, 256, 0));
    if (per_sm < 1) per_sm = 1;
    *warps = per_sm * sm_count * 8;
    return ASYRK_OK;
}

int launch_engine_step(SysDesc *d, int count, int total_chunks, double *part, int resident_warps,
                       bool excl, bool with_outer, cudaStream_t s)
{
    // the server (with_outer) splits half of the warps evenly; a batch, whose
    // members all run to the end of the same iteration, splits by work only
    k_batch_plan<<<1, PLAN_THREADS, 0, s>>>(d, count, resident_warps, with_outer ? 1 : 0);
    ASYRK_CK(cudaGetLastError());
    const unsigned blocks = (unsigned)((resident_warps + 7) / 8);
    if (excl)
        k_batch_project<true><<<blocks, 256, 0, s>>>(d, count);
    else
        k_batch_project<false><<<blocks, 256, 0, s>>>(d, count);
    ASYRK_CK(cudaGetLastError());
    if (total_chunks > 0) {
        k_batch_check<<<(unsigned)total_chunks, 256, 0, s>>>(d, count, part, 0);
        ASYRK_CK(cudaGetLastError());
        if (with_outer) {
            k_batch_outer_update<<<(unsigned)total_chunks, 256, 0, s>>>(d, count);
            ASYRK_CK(cudaGetLastError());
            k_batch_outer_residual<<<(unsigned)total_chunks, 256, 0, s>>>(d, count, part);
            ASYRK_CK(cudaGetLastError());
        }
    }
    return ASYRK_OK;
}

int launch_batch_iteration(SysDesc *d, int count, int total_chunks, double *part,
                           int resident_warps, bool excl, int *d_active, int *d_iter,
                           bool use_cond, unsigned long long cond_handle, cudaStream_t s)
{
    int st = launch_engine_step(d, count, total_chunks, part, resident_warps, excl, false, s);
    if (st != ASYRK_OK) return st;
    k_batch_cond<<<1, 256, 0, s>>>(d, count, d_active, d_iter, use_cond ? 1 : 0,
                                   (cudaGraphConditionalHandle)cond_handle);
    ASYRK_CK(cudaGetLastError());
    return ASYRK_OK;
}

int launch_batch_outer(SysDesc *d, int count, int total_chunks, double *part, cudaStream_t s)
{
    k_batch_outer_update<<<(unsigned)total_chunks, 256, 0, s>>>(d, count);
    ASYRK_CK(cudaGetLastError());
    k_batch_outer_residual<<<(unsigned)total_chunks, 256, 0, s>>>(d, count, part);
    ASYRK_CK(cudaGetLastError());
    return ASYRK_OK;
}

int launch_batch_measure(SysDesc *d, int count, int total_chunks, double *part, cudaStream_t s)
{
    k_batch_check<<<(unsigned)total_chunks, 256, 0, s>>>(d, count, part, 1);
    ASYRK_CK(cudaGetLastError());
    return ASYRK_OK;
}

int launch_batch_residual(SysDesc *d, int count, int total_chunks, double *part, cudaStream_t s)
{
    k_batch_residual<<<(unsigned)total_chunks, 256, 0, s>>>(d, count, part);
    ASYRK_CK(cudaGetLastError());
    return ASYRK_OK;
}

int launch_batch_convert(const double *x64, float *x, int64_t n_total, bool to_f32, cudaStream_t s)
{
    int64_t g = (n_total + 255) / 256;
    if (g > 8192) g = 8192;
    if (g < 1) g = 1;
    if (to_f32)
        k_batch_convert<<<(unsigned)g, 256, 0, s>>>(x64, x, n_total, 1, nullptr, nullptr);
    else
        k_batch_convert<<<(unsigned)g, 256, 0, s>>>(nullptr, nullptr, n_total, 0,
                                                    const_cast<double *>(x64), x);
    ASYRK_CK(cudaGetLastError());
    return ASYRK_OK;
}

int engine_subwarp(const asyrk_problem *p, bool batched)
{
    bool tuned = false;
    int G = tuned_subwarp(p->dtype, p->max_len, p->nnz, p->m, &tuned);
    if (!tuned) G = choose_subwarp(p->max_len, p->nnz, p->m);
    if (!batched) return G;
    return G > 1 ? G / 2 : 1;
}

}  // namespace asyrk
