// cluster.cu -- batched solves with each system's iterate in on-chip memory.
//
// A system whose FP32 iterate x and row-claim bits fit in the shared memory
// of a thread-block cluster of C CTAs (C = 1, 2, 4 or 8) is solved from start
// to finish by one cluster launch:
//   * x is spread over the C CTAs' shared memory, entry t in CTA t mod C at
//     slot t div C (distributed shared memory: every CTA of the cluster reads
//     and updates every slice);
//   * the workers (G lanes each, Section 3's lock-free workers) draw rows from
//     the problem's row sequence exactly as the global-iterate kernels do
//     (Philox counter j, alias table, or shuffled sweeps), stream the row from
//     HBM, gather x from shared memory, and apply Eq. (2)'s full-row update with
//     shared-memory atomic adds (red.shared::cluster.add.f32), so the iterate
//     never travels to L2;
//   * after each sweep (m projections) the cluster meets at a barrier, each
//     CTA reduces its part of the FP64 measure (||x - x*|| and ||x*||, or
//     ||b - A x|| and ||b||), every CTA sums the C parts in rank order and
//     takes the same stop decision (tolerance, divergence, sweep budget);
//   * at the end each CTA writes its slice of x to the FP32 iterate in HBM.
// The number of workers is capped by the Cor. 2 estimate, as in the
// multi-system engine, and by the cluster's threads.  A batch runs one such
// launch per member, all as independent nodes of one CUDA graph.
#include <math.h>
#include <string.h>

#include "batch.cuh"
#include "cluster.cuh"
#include "worker.cuh"

namespace asyrk {

// ---------------------------------------------------------------------------
// shared-memory access: the CTA's own slice (C = 1) or the cluster's slices
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_addr(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned cluster_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// the address of the same shared-memory offset in CTA `rank` of the cluster
__device__ __forceinline__ unsigned map_rank(unsigned a, unsigned rank)
{
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}

__device__ __forceinline__ void cluster_barrier()
{
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

template <bool DS>
__device__ __forceinline__ float sh_ld(unsigned a)
{
    float v;
    if (DS)
        asm volatile("ld.relaxed.cluster.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(a));
    else
        asm volatile("ld.volatile.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}

template <bool DS>
__device__ __forceinline__ void sh_red_add(unsigned a, float v)
{
    if (DS)
        asm volatile("red.relaxed.cluster.shared::cluster.add.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
    else
        asm volatile("red.relaxed.cta.shared.add.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}

template <bool DS>
__device__ __forceinline__ unsigned sh_atom_or(unsigned a, unsigned v)
{
    unsigned old;
    if (DS)
        asm volatile("atom.relaxed.cluster.shared::cluster.or.b32 %0, [%1], %2;"
                     : "=r"(old) : "r"(a), "r"(v) : "memory");
    else
        asm volatile("atom.relaxed.cta.shared.or.b32 %0, [%1], %2;"
                     : "=r"(old) : "r"(a), "r"(v) : "memory");
    return old;
}

template <bool DS>
__device__ __forceinline__ void sh_red_and(unsigned a, unsigned v)
{
    if (DS)
        asm volatile("red.relaxed.cluster.shared::cluster.and.b32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
    else
        asm volatile("red.relaxed.cta.shared.and.b32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

// Where entry t of a distributed array lives: CTA t mod C, slot t div C.
template <bool DS>
struct Slices {
    unsigned base;  // shared-memory address of this CTA's slice
    unsigned mask;  // C - 1
    int lc;         // log2 C
    __device__ __forceinline__ unsigned at(unsigned t) const
    {
        if (!DS) return base + 4u * t;
        return map_rank(base + 4u * (t >> lc), t & mask);
    }
};

template <bool DS>
__device__ __forceinline__ void cl_sync()
{
    if (DS)
        cluster_barrier();
    else
        __syncthreads();
}

// Block sum of two doubles, then the cluster's sum in rank order; every
// thread of every CTA returns the same (t0, t1).
template <bool DS>
__device__ __forceinline__ void cluster_sum2(double v0, double v1, double *wsum, double *cta_part,
                                             double *tot, int C, double &t0, double &t1)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v0 += __shfl_xor_sync(0xffffffffu, v0, o);
        v1 += __shfl_xor_sync(0xffffffffu, v1, o);
    }
    if (lane == 0) {
        wsum[2 * wid] = v0;
        wsum[2 * wid + 1] = v1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < nw; ++w) {
            a += wsum[2 * w];
            b += wsum[2 * w + 1];
        }
        cta_part[0] = a;
        cta_part[1] = b;
    }
    cl_sync<DS>();  // every CTA's part is written
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        const unsigned pa = smem_addr(cta_part);
        for (int r = 0; r < C; ++r) {
            double x0, x1;
            if (DS) {
                const unsigned q = map_rank(pa, (unsigned)r);
                asm volatile("ld.relaxed.cluster.shared::cluster.f64 %0, [%1];" : "=d"(x0) : "r"(q) : "memory");
                asm volatile("ld.relaxed.cluster.shared::cluster.f64 %0, [%1];" : "=d"(x1) : "r"(q + 8u) : "memory");
            } else {
                x0 = cta_part[0];
                x1 = cta_part[1];
            }
            a += x0;
            b += x1;
        }
        tot[0] = a;
        tot[1] = b;
    }
    __syncthreads();
    t0 = tot[0];
    t1 = tot[1];
}

__device__ __forceinline__ double entry_f64(const float *v, long long k) { return (double)v[k]; }
__device__ __forceinline__ double entry_f64(const bf16_t *v, long long k)
{
    return (double)__uint_as_float(((unsigned)v[k].bits) << 16);
}

// The FP64 measure of the cluster's current x: (||x - x*||^2, ||x*||^2) when
// err_form, else (||b - A x||^2, ||b||^2) with b at FP32 -- the row records'
// b, or bvec (a refinement's right-hand side) when given.
template <typename VT, bool DS>
__device__ __forceinline__ void cluster_measure(const ClusterJob &J, const Slices<DS> &X,
                                                const float *xs, unsigned rank, int C,
                                                bool err_form, const float *bvec, double *wsum,
                                                double *cta_part, double *tot, double &t0,
                                                double &t1)
{
    double v0 = 0.0, v1 = 0.0;
    const int T = (int)blockDim.x;
    if (err_form) {
        const int nper = J.nper;
        for (int o = threadIdx.x; o < nper; o += T) {
            const long long t = ((long long)o << J.lc) + rank;
            if (t < J.n) {
                const double xt = J.xt[t];
                const double e = (double)sh_ld<false>(smem_addr(xs + o)) - xt;
                v0 += e * e;
                v1 += xt * xt;
            }
        }
    } else {
        const VT *val = static_cast<const VT *>(J.val);
        for (long long i = (long long)rank * T + threadIdx.x; i < J.m; i += (long long)C * T) {
            const RowRec r = load_rec(J.rec + i);
            double acc = 0.0;
            for (unsigned q = 0; q < r.len; ++q)
                acc += entry_f64(val, r.start + q) *
                       (double)sh_ld<DS>(X.at((unsigned)J.col[r.start + q]));
            const double bi = bvec ? (double)__ldcg(bvec + i) : (double)r.b;
            const double ri = bi - acc;
            v0 += ri * ri;
            v1 += bi * bi;
        }
    }
    cluster_sum2<DS>(v0, v1, wsum, cta_part, tot, C, t0, t1);
}

// The outer step of mixed-precision refinement: x64 += d and d = 0 over this
// CTA's entries; then, with every CTA's update in place, r = b - A x64 in FP64
// over the cluster's rows, stored at FP32 in r32 (the next inner solve's
// right-hand side).  Returns (||r||^2, ||x64 - x*||^2) (the latter 0 without x*).
template <typename VT, bool DS>
__device__ __forceinline__ void cluster_outer(const ClusterJob &J, float *xs, unsigned rank, int C,
                                              double *wsum, double *cta_part, double *tot,
                                              double &t0, double &t1)
{
    const int T = (int)blockDim.x;
    for (int o = threadIdx.x; o < J.nper; o += T) {
        const long long t = ((long long)o << J.lc) + rank;
        if (t < J.n) J.x64[t] = __ldcg(J.x64 + t) + (double)xs[o];
        xs[o] = 0.f;
    }
    cl_sync<DS>();  // x64 complete
    double v0 = 0.0, v1 = 0.0;
    const VT *val = static_cast<const VT *>(J.val);
    for (long long i = (long long)rank * T + threadIdx.x; i < J.m; i += (long long)C * T) {
        const RowRec r = load_rec(J.rec + i);
        double acc = 0.0;
        for (unsigned q = 0; q < r.len; ++q)
            acc += entry_f64(val, r.start + q) * __ldcg(J.x64 + J.col[r.start + q]);
        const double ri = J.b64[i] - acc;
        J.r32[i] = (float)ri;
        v0 += ri * ri;
    }
    if (J.xt) {
        for (int o = threadIdx.x; o < J.nper; o += T) {
            const long long t = ((long long)o << J.lc) + rank;
            if (t < J.n) {
                const double e = __ldcg(J.x64 + t) - J.xt[t];
                v1 += e * e;
            }
        }
    }
    cluster_sum2<DS>(v0, v1, wsum, cta_part, tot, C, t0, t1);
}

// A solve's progress, kept in shared memory (thread 0 of each CTA writes it).
struct SolveState {
    double meas, meas0;  // last and first measure
    double ref_in;       // refinement: ||r|| of the current inner solve
    double res2;         // refinement: ||b - A x64||^2 of the last outer step
    double inner_goal;   // refinement: this outer step's inner target
    double rprev;        // refinement: ||r|| of the previous outer step (< 0: none)
    long long inner_plan;  // refinement: inner sweeps this outer step runs
    long long sweeps, inner_sweeps;
    int status, outer_steps;
    int done, outer_next;
};

// First half of the row draw of projection j (the global kernels' draw_row):
// the Philox words at counter (j_lo, j_hi, stream, 0), the bucket floor(u0 m / 2^32)
// and its record; `coin` = u1 decides the alias later.  Shuffled sweeps: the
// row pi_k(j mod m) and its record, no alias.
__device__ __forceinline__ void prefetch_draw(unsigned long long j, const ClusterJob &J,
                                              const RowRec *rec, unsigned m, unsigned &i,
                                              unsigned &coin, RowRec &r)
{
    if (J.sampling == 1) {
        i = shuffled_position(j, m, J.stream_id, J.key, J.shuf_h);
        coin = 0u;
    } else {
        const uint4 u = philox4x32_10(make_uint4((unsigned)j, (unsigned)(j >> 32), J.stream_id, 0u),
                                      J.key);
        i = __umulhi(u.x, m);
        coin = u.y;
    }
    r = load_rec(rec + i);
}

template <typename VT, int G, bool DS>
__device__ __forceinline__ void cluster_solve(ClusterJob *jobs, int k)
{
    extern __shared__ __align__(16) unsigned char cl_dyn[];
    __shared__ double wsum[2 * (CLUSTER_MAX_THREADS / 32)];
    __shared__ double cta_part[2];
    __shared__ double tot[2];
    __shared__ unsigned long long cta_skipped;
    __shared__ ClusterJob sj;  // the job's fields, read from shared memory in the loops
    __shared__ SolveState ss;

    if (threadIdx.x == 0) sj = jobs[k];
    __syncthreads();
    const ClusterJob &J = sj;
    const unsigned rank = DS ? cluster_rank() : 0u;
    const int lc = J.lc, C = 1 << lc;
    const int T = (int)blockDim.x;
    float *xs = reinterpret_cast<float *>(cl_dyn);
    unsigned *bs = reinterpret_cast<unsigned *>(cl_dyn + 4 * (size_t)J.nper_pad);
    const Slices<DS> X{smem_addr(xs), (unsigned)(C - 1), lc};
    const Slices<DS> B{smem_addr(bs), (unsigned)(C - 1), lc};

    // 1. this CTA's slice of the shared iterate -- x0 from the FP64 iterate, or
    // for refinement the correction d = 0 -- and the claim bits cleared
    const bool refine = J.refine != 0;
    for (int o = threadIdx.x; o < J.nper; o += T) {
        const long long t = ((long long)o << lc) + rank;
        xs[o] = (t < J.n && !refine) ? (float)J.x64[t] : 0.f;
    }
    for (int o = threadIdx.x; o < J.bper; o += T) bs[o] = 0u;
    if (threadIdx.x == 0) cta_skipped = 0ull;
    cl_sync<DS>();  // all slices initialised (and, in a cluster, every CTA running)

    // 2. the first measure: ||x0 - x*|| / ||x*|| (or the residual); with
    // refinement only ||x*|| (the outer measure's reference), the outer step
    // measures the rest.  The solve's state lives in shared memory: thread 0
    // of each CTA takes the decisions (every CTA from the same sums), every
    // thread reads them after the next barrier.
    double t0, t1;
    cluster_measure<VT, DS>(J, X, xs, rank, C, J.xt != nullptr, nullptr, wsum, cta_part, tot, t0, t1);
    const double ref = J.xt ? (sqrt(t1) > 0.0 ? sqrt(t1) : 1.0) : (J.bnorm > 0.0 ? J.bnorm : 1.0);
    if (threadIdx.x == 0) {
        ss.meas = ss.meas0 = -1.0;
        ss.ref_in = 1.0;
        ss.res2 = 0.0;
        ss.inner_goal = J.inner_tol;
        ss.rprev = -1.0;
        ss.inner_plan = J.max_inner < 8 ? (J.max_inner > 0 ? J.max_inner : 1) : 8;
        ss.status = ASYRK_NOT_CONVERGED;
        ss.outer_steps = 0;
        ss.inner_sweeps = 0;
        ss.sweeps = 0;
        ss.done = 0;
        ss.outer_next = refine ? 1 : 0;
        if (!refine) {
            ss.meas = ss.meas0 = sqrt(t0) / ref;
            if (ss.meas <= J.tol) {
                ss.status = ASYRK_OK;
                ss.done = 1;
            } else if (J.max_sweeps <= 0) {
                ss.done = 1;
            }
        }
    }
    __syncthreads();
    const float *bvec = refine ? J.r32 : nullptr;

    // worker layout: cluster thread id -> worker (G lanes of one warp)
    const int lane = threadIdx.x & 31;
    const int sub = lane / G, sl = lane % G;
    const long long warp_first = ((long long)rank * T + threadIdx.x) / 32 * (32 / G);
    const long long W = J.workers;
    const bool worker = warp_first + sub < W;
    const VT *__restrict__ val = static_cast<const VT *>(J.val);
    const int32_t *__restrict__ col = J.col;
    const RowRec *__restrict__ rec = J.rec;
    const float gamma = J.gamma;
    const unsigned m = J.m;
    const bool excl = J.excl != 0;
    const bool seq = W == 1;
    unsigned long long skipped = 0;

    // 3. sweeps until the measure meets the tolerance (or diverges, or the budget
    // ends); with refinement, outer steps r = b - A x64, x64 += d between inner
    // solves of A d = r (the multi-system engine's refinement, in one CTA)
    for (;;) {
        if (ss.done) break;
        if (ss.outer_next) {
            cluster_outer<VT, DS>(J, xs, rank, C, wsum, cta_part, tot, t0, t1);
            if (threadIdx.x == 0) {
                const double rnorm = sqrt(t0);
                const double meas = J.xt ? sqrt(t1) / ref : rnorm / ref;
                ss.meas = meas;
                if (ss.meas0 < 0.0) ss.meas0 = meas;
                ss.outer_steps += 1;
                ss.res2 = t0;
                if (!isfinite(meas) || meas > 1e30 * (ss.meas0 > 0.0 ? ss.meas0 : 1.0)) {
                    ss.status = ASYRK_DIVERGED;
                    ss.done = 1;
                } else if (meas <= J.tol || rnorm == 0.0) {
                    ss.status = ASYRK_OK;
                    ss.done = 1;
                } else if (ss.sweeps >= J.max_sweeps) {
                    ss.done = 1;
                }
                ss.outer_next = 0;
                ss.ref_in = rnorm;
                ss.inner_sweeps = 0;
                ss.inner_goal = refine_inner_goal(J.inner_tol, J.tol, meas);
                // the inner sweep count, as single solves plan it: from the
                // contraction the last step's sweeps achieved, the count that
                // meets this step's target (at least 2, at most 4x the last)
                if (ss.rprev > 0.0 && rnorm > 0.0) {
                    const double rho = rnorm / ss.rprev;
                    long long inner = ss.inner_plan;
                    if (rho > 0.0 && rho < 1.0) {
                        double want = (double)inner * log(ss.inner_goal) / log(rho);
                        if (want < 2.0) want = 2.0;
                        if (want > 4.0 * (double)inner) want = 4.0 * (double)inner;
                        inner = (long long)ceil(want);
                    } else {
                        inner *= 2;
                    }
                    if (inner > J.max_inner) inner = J.max_inner;
                    ss.inner_plan = inner > 0 ? inner : 1;
                }
                ss.rprev = rnorm;
            }
            cl_sync<DS>();  // r32 complete before the inner solve reads it; decisions visible
            continue;
        }
        const long long sweeps = ss.sweeps;
        const unsigned long long jbase = J.j0 + (unsigned long long)sweeps * m;
        if (warp_first < W) {
            // The draw is split in two so that the record load of a worker's next
            // projection is in flight while it works on the current one: the
            // prefetch computes the Philox words and loads the bucket's record (or,
            // for shuffled sweeps, the row's); at its turn the projection takes the
            // bucket's alias when the coin says so (a second, dependent load).
            bool nact = worker && (unsigned long long)warp_first + sub < m;
            unsigned ni = 0, ncoin = 0;
            RowRec nr{};
            if (nact) prefetch_draw(jbase + warp_first + sub, J, rec, m, ni, ncoin, nr);
            for (unsigned long long t0w = (unsigned long long)warp_first; t0w < m;
                 t0w += (unsigned long long)W) {
                const unsigned long long t = t0w + sub;
                bool act = nact;
                unsigned i = ni;
                RowRec r = nr;
                if (act && J.sampling == 0 && !J.uniform && ncoin >= r.thr) {
                    i = r.alias;
                    r = load_rec(rec + i);
                }
                const long long start = act ? r.start : 0;
                int len = act ? (int)r.len : 0;
                const float b = (bvec && act) ? __ldcg(bvec + i) : r.b, scale = r.inv;
                // a lane's first two chunks of 4 entries (rows up to 8G entries) stay
                // in registers from the dot product to the update (one chunk when a
                // single lane walks the row); their loads go out before the next
                // draw's Philox work, which then runs while they are in flight
                int4 cc, cc1;
                float vv[4], vv1[4];
                const int off0 = sl * 4, off1 = G > 1 ? (G + sl) * 4 : 0x7fffffff;
                const int tail0 = ((G > 1 ? 2 * G : G) + sl) * 4;
                if (off0 < len) {
                    cc = ld_col4(col + start + off0);
                    ld_val4(val + start + off0, vv);
                }
                if (off1 < len) {
                    cc1 = ld_col4(col + start + off1);
                    ld_val4(val + start + off1, vv1);
                }
                nact = worker && t + (unsigned long long)W < m;
                if (nact) prefetch_draw(jbase + t + W, J, rec, m, ni, ncoin, nr);
                if (excl) {
                    unsigned got = 0;
                    if (act && sl == 0) {
                        const unsigned bit = 1u << (i & 31);
                        got = !(sh_atom_or<DS>(B.at(i >> 5), bit) & bit);
                    }
                    got = __shfl_sync(0xffffffffu, got, lane & ~(G - 1));
                    if (act && !got) {
                        act = false;
                        len = 0;
                        if (sl == 0) ++skipped;
                    }
                }
                float acc = 0.f;
                if (off0 < len) {
                    const int kk = len - off0;
                    acc = vv[0] * sh_ld<DS>(X.at((unsigned)cc.x));
                    if (kk > 1) acc += vv[1] * sh_ld<DS>(X.at((unsigned)cc.y));
                    if (kk > 2) acc += vv[2] * sh_ld<DS>(X.at((unsigned)cc.z));
                    if (kk > 3) acc += vv[3] * sh_ld<DS>(X.at((unsigned)cc.w));
                }
                if (off1 < len) {
                    const int kk = len - off1;
                    acc += vv1[0] * sh_ld<DS>(X.at((unsigned)cc1.x));
                    if (kk > 1) acc += vv1[1] * sh_ld<DS>(X.at((unsigned)cc1.y));
                    if (kk > 2) acc += vv1[2] * sh_ld<DS>(X.at((unsigned)cc1.z));
                    if (kk > 3) acc += vv1[3] * sh_ld<DS>(X.at((unsigned)cc1.w));
                }
                for (int off = tail0; off < len; off += 4 * G) {  // rows longer than 8G (4 for G = 1)
                    float v4[4];
                    const int4 c4 = ld_col4(col + start + off);
                    ld_val4(val + start + off, v4);
                    const int kk = len - off;
                    acc += v4[0] * sh_ld<DS>(X.at((unsigned)c4.x));
                    if (kk > 1) acc += v4[1] * sh_ld<DS>(X.at((unsigned)c4.y));
                    if (kk > 2) acc += v4[2] * sh_ld<DS>(X.at((unsigned)c4.z));
                    if (kk > 3) acc += v4[3] * sh_ld<DS>(X.at((unsigned)c4.w));
                }
#pragma unroll
                for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (act) {
                    const float s = -(gamma * (acc - b) * scale);
                    if (off0 < len) {
                        const int kk = len - off0;
                        sh_red_add<DS>(X.at((unsigned)cc.x), s * vv[0]);
                        if (kk > 1) sh_red_add<DS>(X.at((unsigned)cc.y), s * vv[1]);
                        if (kk > 2) sh_red_add<DS>(X.at((unsigned)cc.z), s * vv[2]);
                        if (kk > 3) sh_red_add<DS>(X.at((unsigned)cc.w), s * vv[3]);
                    }
                    if (off1 < len) {
                        const int kk = len - off1;
                        sh_red_add<DS>(X.at((unsigned)cc1.x), s * vv1[0]);
                        if (kk > 1) sh_red_add<DS>(X.at((unsigned)cc1.y), s * vv1[1]);
                        if (kk > 2) sh_red_add<DS>(X.at((unsigned)cc1.z), s * vv1[2]);
                        if (kk > 3) sh_red_add<DS>(X.at((unsigned)cc1.w), s * vv1[3]);
                    }
                    for (int off = tail0; off < len; off += 4 * G) {
                        float v4[4];
                        const int4 c4 = ld_col4(col + start + off);
                        ld_val4(val + start + off, v4);
                        const int kk = len - off;
                        sh_red_add<DS>(X.at((unsigned)c4.x), s * v4[0]);
                        if (kk > 1) sh_red_add<DS>(X.at((unsigned)c4.y), s * v4[1]);
                        if (kk > 2) sh_red_add<DS>(X.at((unsigned)c4.z), s * v4[2]);
                        if (kk > 3) sh_red_add<DS>(X.at((unsigned)c4.w), s * v4[3]);
                    }
                }
                if (excl) {
                    __syncwarp();  // the group's updates are issued before the bit is cleared
                    if (act && sl == 0) sh_red_and<DS>(B.at(i >> 5), ~(1u << (i & 31)));
                }
                if (seq) {  // one worker: each update lands before the next gather
                    if (DS)
                        asm volatile("fence.acq_rel.cluster;" ::: "memory");
                    else
                        __threadfence_block();
                    __syncwarp();
                }
            }
        }
        cl_sync<DS>();  // the sweep's updates are all applied
        // inner solves run their planned sweeps unmeasured (the outer step
        // measures); plain solves measure every sweep
        if (!refine)
            cluster_measure<VT, DS>(J, X, xs, rank, C, J.xt != nullptr, bvec, wsum, cta_part,
                                    tot, t0, t1);
        if (threadIdx.x == 0) {
            ss.sweeps = sweeps + 1;
            if (refine) {
                ss.inner_sweeps += 1;
                if (ss.inner_sweeps >= ss.inner_plan || ss.inner_sweeps >= J.max_inner ||
                    ss.sweeps >= J.max_sweeps)
                    ss.outer_next = 1;
            } else {
                const double meas = sqrt(t0) / ref;
                ss.meas = meas;
                if (!isfinite(meas) || meas > 1e30 * (ss.meas0 > 0.0 ? ss.meas0 : 1.0)) {
                    ss.status = ASYRK_DIVERGED;
                    ss.done = 1;
                } else if (meas <= J.tol) {
                    ss.status = ASYRK_OK;
                    ss.done = 1;
                } else if (ss.sweeps >= J.max_sweeps) {
                    ss.done = 1;
                }
            }
        }
        cl_sync<DS>();  // decisions visible; no CTA starts the next sweep while another measures
    }

    // 4. results: x to the FP32 iterate in HBM (refinement: x64 holds the
    // iterate, the last outer step folded d into it), counters
    for (int o = threadIdx.x; o < J.nper && !refine; o += T) {
        const long long t = ((long long)o << lc) + rank;
        if (t < J.n) J.x32[t] = xs[o];
    }
    if (skipped) atomicAdd(&cta_skipped, skipped);
    __syncthreads();
    ClusterJob &Jw = jobs[k];
    if (threadIdx.x == 0) {
        if (cta_skipped) atomicAdd(&Jw.skipped, cta_skipped);
        if (rank == 0) {
            Jw.meas = ss.meas;
            Jw.meas0 = ss.meas0;
            Jw.sweeps = ss.sweeps;
            Jw.status = ss.status;
            Jw.outer_steps = ss.outer_steps;
            Jw.res2 = ss.res2;
        }
    }
    cl_sync<DS>();  // no CTA leaves while another may still read its shared memory
}

// one member's solve: jobs[k] (a cluster of C CTAs, or one CTA)
template <typename VT, int G, bool DS>
__global__ void __launch_bounds__(CLUSTER_MAX_THREADS, 1) k_cluster_solve(ClusterJob *jobs, int k)
{
    cluster_solve<VT, G, DS>(jobs, k);
}

// many one-CTA members in one launch: CTA b solves jobs[list[b]]
template <typename VT, int G>
__global__ void __launch_bounds__(CLUSTER_MAX_THREADS, 1)
    k_cluster_solve_list(ClusterJob *jobs, const int *__restrict__ list)
{
    cluster_solve<VT, G, false>(jobs, list[blockIdx.x]);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
using ClusterKernel = void (*)(ClusterJob *, int);

template <typename VT, bool DS>
static ClusterKernel pick_g(int G)
{
    switch (G) {
    case 1: return k_cluster_solve<VT, 1, DS>;
    case 2: return k_cluster_solve<VT, 2, DS>;
    case 4: return k_cluster_solve<VT, 4, DS>;
    case 8: return k_cluster_solve<VT, 8, DS>;
    case 16: return k_cluster_solve<VT, 16, DS>;
    case 32: return k_cluster_solve<VT, 32, DS>;
    default: return nullptr;
    }
}

static ClusterKernel pick_kernel(int dtype, int G, bool ds)
{
    if (dtype == ASYRK_F32) return ds ? pick_g<float, true>(G) : pick_g<float, false>(G);
    if (dtype == ASYRK_BF16) return ds ? pick_g<bf16_t, true>(G) : pick_g<bf16_t, false>(G);
    return nullptr;
}

static size_t dyn_bytes(int64_t n, int64_t m, int C, int *nper, int *nper_pad, int *bper)
{
    const int64_t np = (n + C - 1) / C;
    const int64_t words = (m + 31) / 32;
    const int64_t bp = (words + C - 1) / C;
    const int64_t npad = (np + 3) & ~(int64_t)3;  // claim words start 16-byte aligned
    *nper = (int)np;
    *nper_pad = (int)npad;
    *bper = (int)bp;
    return (size_t)(4 * npad + 4 * bp);
}

int cluster_shape(const asyrk_problem *p, int G, int cluster_max, int max_workers,
                  ClusterShape *sh)
{
    memset(sh, 0, sizeof *sh);
    if (p->dtype != ASYRK_F32 && p->dtype != ASYRK_BF16) return ASYRK_OK;  // does not fit
    if (p->m > 0x7fffffffLL || p->n > 0x7fffffffLL) return ASYRK_OK;
    if (cluster_max < 1) cluster_max = CLUSTER_DEFAULT_MAX;
    if (cluster_max > CLUSTER_MAX_SIZE) cluster_max = CLUSTER_MAX_SIZE;
    long long cap = tau_cap_estimate(p->m, p->n);
    if (max_workers > 0 && max_workers < cap) cap = max_workers;
    // the smallest cluster whose shared memory holds the system ...
    int C = 1, nper = 0, npad = 0, bper = 0;
    size_t bytes = dyn_bytes(p->n, p->m, C, &nper, &npad, &bper);
    while (bytes > CLUSTER_SMEM_BYTES && C < cluster_max) {
        C *= 2;
        bytes = dyn_bytes(p->n, p->m, C, &nper, &npad, &bper);
    }
    if (bytes > CLUSTER_SMEM_BYTES) return ASYRK_OK;  // does not fit
    // ... grown while the Cor. 2 worker cap asks for more threads than it has
    while (C < cluster_max && (long long)cap * G > (long long)C * CLUSTER_MAX_THREADS) {
        C *= 2;
        bytes = dyn_bytes(p->n, p->m, C, &nper, &npad, &bper);
    }
    long long thr = (cap * G + C - 1) / C;
    thr = (thr + 31) / 32 * 32;
    if (thr > CLUSTER_MAX_THREADS) thr = CLUSTER_MAX_THREADS;
    if (thr < 32) thr = 32;
    long long W = (long long)C * thr / G;
    if (W > cap) W = cap;
    sh->fits = 1;
    sh->C = C;
    sh->lc = 0;
    while ((1 << sh->lc) < C) ++sh->lc;
    sh->threads = (int)thr;
    sh->workers = (int)W;
    sh->G = G;
    sh->smem = bytes;
    sh->nper = nper;
    sh->nper_pad = npad;
    sh->bper = bper;
    return ASYRK_OK;
}

int cluster_prepare(int dtype, int G, int C)
{
    ClusterKernel k = pick_kernel(dtype, G, C > 1);
    if (!k) return set_error(ASYRK_EINVAL, "no on-chip kernel for dtype %d, subwarp %d", dtype, G);
    ASYRK_CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)CLUSTER_SMEM_BYTES));
    return ASYRK_OK;
}

int cluster_check_schedulable(int dtype, const ClusterShape &sh)
{
    ClusterKernel k = pick_kernel(dtype, sh.G, sh.C > 1);
    if (!k) return set_error(ASYRK_EINVAL, "no on-chip kernel for subwarp %d", sh.G);
    if (sh.C == 1) {
        int per_sm = 0;
        ASYRK_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, sh.threads, sh.smem));
        if (per_sm < 1)
            return set_error(ASYRK_EINVAL, "on-chip shape (%d threads, %zu B) does not fit an SM",
                             sh.threads, sh.smem);
        return ASYRK_OK;
    }
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.gridDim = dim3((unsigned)sh.C);
    cfg.blockDim = dim3((unsigned)sh.threads);
    cfg.dynamicSmemBytes = sh.smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)sh.C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int clusters = 0;
    ASYRK_CK(cudaOccupancyMaxActiveClusters(&clusters, (void *)k, &cfg));
    if (clusters < 1)
        return set_error(ASYRK_EINVAL, "on-chip cluster of %d CTAs (%d threads, %zu B) cannot be scheduled",
                         sh.C, sh.threads, sh.smem);
    return ASYRK_OK;
}

int cluster_add_node(cudaGraph_t g, int dtype, const ClusterShape &sh, ClusterJob *jobs, int k)
{
    ClusterKernel fn = pick_kernel(dtype, sh.G, sh.C > 1);
    if (!fn) return set_error(ASYRK_EINVAL, "no on-chip kernel for subwarp %d", sh.G);
    void *args[2] = {&jobs, &k};
    cudaKernelNodeParams kp;
    memset(&kp, 0, sizeof kp);
    kp.func = (void *)fn;
    kp.gridDim = dim3((unsigned)sh.C);
    kp.blockDim = dim3((unsigned)sh.threads);
    kp.sharedMemBytes = (unsigned)sh.smem;
    kp.kernelParams = args;
    cudaGraphNode_t node;
    ASYRK_CK(cudaGraphAddKernelNode(&node, g, nullptr, 0, &kp));
    if (sh.C > 1) {
        cudaLaunchAttributeValue v;
        memset(&v, 0, sizeof v);
        v.clusterDim.x = (unsigned)sh.C;
        v.clusterDim.y = 1;
        v.clusterDim.z = 1;
        ASYRK_CK(cudaGraphKernelNodeSetAttribute(node, cudaLaunchAttributeClusterDimension, &v));
    }
    return ASYRK_OK;
}

using ClusterListKernel = void (*)(ClusterJob *, const int *);

template <typename VT>
static ClusterListKernel pick_list_g(int G)
{
    switch (G) {
    case 1: return k_cluster_solve_list<VT, 1>;
    case 2: return k_cluster_solve_list<VT, 2>;
    case 4: return k_cluster_solve_list<VT, 4>;
    case 8: return k_cluster_solve_list<VT, 8>;
    case 16: return k_cluster_solve_list<VT, 16>;
    case 32: return k_cluster_solve_list<VT, 32>;
    default: return nullptr;
    }
}

int cluster_add_list_node(cudaGraph_t g, int dtype, int G, int threads, size_t smem, int ctas,
                          ClusterJob *jobs, const int *list)
{
    ClusterListKernel fn = dtype == ASYRK_BF16 ? pick_list_g<bf16_t>(G) : pick_list_g<float>(G);
    if (!fn || ctas < 1) return set_error(ASYRK_EINVAL, "no on-chip kernel for subwarp %d", G);
    if (smem > 48 * 1024) {
        ASYRK_CK(cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)CLUSTER_SMEM_BYTES));
    }
    void *args[2] = {&jobs, &list};
    cudaKernelNodeParams kp;
    memset(&kp, 0, sizeof kp);
    kp.func = (void *)fn;
    kp.gridDim = dim3((unsigned)ctas);
    kp.blockDim = dim3((unsigned)threads);
    kp.sharedMemBytes = (unsigned)smem;
    kp.kernelParams = args;
    cudaGraphNode_t node;
    ASYRK_CK(cudaGraphAddKernelNode(&node, g, nullptr, 0, &kp));
    return ASYRK_OK;
}

int cluster_launch(int dtype, const ClusterShape &sh, ClusterJob *jobs, int k, cudaStream_t s)
{
    ClusterKernel fn = pick_kernel(dtype, sh.G, sh.C > 1);
    if (!fn) return set_error(ASYRK_EINVAL, "no on-chip kernel for subwarp %d", sh.G);
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.gridDim = dim3((unsigned)sh.C);
    cfg.blockDim = dim3((unsigned)sh.threads);
    cfg.dynamicSmemBytes = sh.smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)sh.C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = sh.C > 1 ? 1 : 0;
    ASYRK_CK(cudaLaunchKernelEx(&cfg, fn, jobs, k));
    return ASYRK_OK;
}

}  // namespace asyrk
