// project.cu -- the row-projection kernels (the method's hot loop).
//
// One "worker" is a group of G lanes of a warp (G = 2..32), so a warp runs
// 32/G workers side by side.  Worker w applies projections t = w, w + W,
// w + 2W, ... of the launch (W = number of workers), projection t being
// number j = j0 + t of the problem's row sequence.  For each projection
// (Section 3's five per-thread steps, with the full-row update of
// Section 5):
//   1. draw the row i (Philox counter j, alias table; one 32-byte record);
//   2. load the row's columns and values, 4 per lane with 16-byte loads;
//   3. gather x on supp(a_i) from L2 and reduce a_i^T x across the G lanes;
//   4. s = -gamma (a_i^T x - b_i) / ||a_i||^2;
//   5. x_t += s * A_it for every t in supp(a_i), each as one red.global.add
//      (an atomic add that returns nothing; no locks, Section 3).
// Reads of x are not synchronised with other workers' updates, so a worker
// may project with an x that misses up to about W - 1 concurrent updates:
// the staleness bound tau of Eq. (4) is set by W.
//
// With sequential = true a single worker (one warp) applies the projections
// strictly in order, fencing its updates before the next gather: the
// sequential RK iterate of Eq. (2).
#include <type_traits>

#include "common.cuh"

namespace asyrk {

struct ProjArgs {
    const RowRec *rec;
    const int32_t *col;
    const void *val;
    void *x;
    const double *b64;
    const double *w64;
    uint2 key;
    unsigned m;
    int uniform;
    unsigned stream_id;
    unsigned long long j0;
    unsigned long long count;
    long long workers;
    double gamma;
    unsigned *busy;                  // row-claim bits (row exclusion)
    unsigned long long *skipped;     // projections skipped by row exclusion
};

// ---- streamed row loads: read once per projection, so marked evict-first --
__device__ __forceinline__ int4 ld_col4(const int32_t *p)
{
    return __ldcs(reinterpret_cast<const int4 *>(p));
}

template <typename XT>
__device__ __forceinline__ void ld_val4(const double *p, XT (&v)[4])
{
    const double2 a = __ldcs(reinterpret_cast<const double2 *>(p));
    const double2 b = __ldcs(reinterpret_cast<const double2 *>(p) + 1);
    v[0] = (XT)a.x; v[1] = (XT)a.y; v[2] = (XT)b.x; v[3] = (XT)b.y;
}

template <typename XT>
__device__ __forceinline__ void ld_val4(const float *p, XT (&v)[4])
{
    const float4 a = __ldcs(reinterpret_cast<const float4 *>(p));
    v[0] = (XT)a.x; v[1] = (XT)a.y; v[2] = (XT)a.z; v[3] = (XT)a.w;
}

template <typename XT>
__device__ __forceinline__ void ld_val4(const bf16_t *p, XT (&v)[4])
{
    const uint2 a = __ldcs(reinterpret_cast<const uint2 *>(p));
    v[0] = (XT)__uint_as_float(a.x << 16);
    v[1] = (XT)__uint_as_float(a.x & 0xffff0000u);
    v[2] = (XT)__uint_as_float(a.y << 16);
    v[3] = (XT)__uint_as_float(a.y & 0xffff0000u);
}

// ---- the shared iterate: gathers from L2 (no L1 copy that could go stale
// for longer than the updates in flight), updates as reductions at L2 ------
__device__ __forceinline__ float ld_x(const float *p) { return __ldcg(p); }
__device__ __forceinline__ double ld_x(const double *p) { return __ldcg(p); }

__device__ __forceinline__ void red_add(float *p, float v)
{
    asm volatile("red.relaxed.gpu.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}
__device__ __forceinline__ void red_add(double *p, double v)
{
    asm volatile("red.relaxed.gpu.global.add.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}

template <typename XT>
__device__ __forceinline__ XT dot4(const XT (&v)[4], int4 c, int k, const XT *x)
{
    // k = entries of this chunk that belong to the row (>= 1)
    XT acc = v[0] * ld_x(x + c.x);
    if (k > 1) acc += v[1] * ld_x(x + c.y);
    if (k > 2) acc += v[2] * ld_x(x + c.z);
    if (k > 3) acc += v[3] * ld_x(x + c.w);
    return acc;
}

template <typename XT>
__device__ __forceinline__ void scatter4(const XT (&v)[4], int4 c, int k, XT s, XT *x)
{
    red_add(x + c.x, s * v[0]);
    if (k > 1) red_add(x + c.y, s * v[1]);
    if (k > 2) red_add(x + c.z, s * v[2]);
    if (k > 3) red_add(x + c.w, s * v[3]);
}

// Row exclusion: a worker claims its row in a bitmask (one bit per row, at
// L2) with an acquire atomic OR before gathering x, and releases it with a
// release AND after its updates.  A row already claimed is skipped: no row is
// ever applied twice from the same stale x, the property the paper's
// implementation gets from giving each thread its own rows (Section 5).  The
// skipped projection would, in the sequential order, come right after the
// same projection and change x only through the few updates in between
// (projections are idempotent).
__device__ __forceinline__ unsigned claim_row(unsigned *busy, unsigned i)
{
    unsigned old;
    asm volatile("atom.acquire.gpu.global.or.b32 %0, [%1], %2;"
                 : "=r"(old)
                 : "l"(busy + (i >> 5)), "r"(1u << (i & 31))
                 : "memory");
    return !(old & (1u << (i & 31)));
}

__device__ __forceinline__ void release_row(unsigned *busy, unsigned i)
{
    asm volatile("red.release.gpu.global.and.b32 [%0], %1;" ::"l"(busy + (i >> 5)),
                 "r"(~(1u << (i & 31)))
                 : "memory");
}

template <typename VT, typename XT, int G, bool SEQ, bool EXCL>
__global__ void __launch_bounds__(256) k_project(const ProjArgs a)
{
    constexpr int GPW = 32 / G;  // workers per warp
    constexpr int CH = 2;        // row chunks of 4G entries kept in registers
    constexpr bool F64 = std::is_same<XT, double>::value;
    const int lane = threadIdx.x & 31;
    const int sub = lane / G, sl = lane % G;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long W = a.workers;
    const long long gbase = warp * GPW;
    if (gbase >= W) return;  // whole warp idle
    const bool worker = gbase + sub < W;
    const VT *__restrict__ val = static_cast<const VT *>(a.val);
    XT *x = static_cast<XT *>(a.x);
    const XT gamma = (XT)a.gamma;
    unsigned long long skipped = 0;

    // t0 walks k*W + gbase, so worker gbase+sub gets projection t0 + sub.  The
    // trip count is warp-uniform: every lane reaches every shuffle and barrier.
    for (unsigned long long t0 = (unsigned long long)gbase; t0 < a.count;
         t0 += (unsigned long long)W) {
        const unsigned long long t = t0 + sub;
        bool act = worker && t < a.count;
        long long start = 0;
        int len = 0;
        unsigned i = 0;
        XT b = 0, scale = 0;
        if (act) {
            RowRec r;
            i = draw_row(a.j0 + t, a.stream_id, a.key, a.m, a.uniform, a.rec, r);
            start = r.start;
            len = (int)r.len;
            if (F64) {
                b = (XT)__ldg(a.b64 + i);
                scale = (XT)__ldg(a.w64 + i);
            } else {
                b = (XT)r.b;
                scale = (XT)r.inv;
            }
        }
        int4 cc[CH];
        XT vv[CH][4];
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const int off = (c * G + sl) * 4;
            if (off < len) {
                cc[c] = ld_col4(a.col + start + off);
                ld_val4(val + start + off, vv[c]);
            }
        }
        if (EXCL) {
            unsigned got = 0;
            if (act && sl == 0) got = claim_row(a.busy, i);
            __syncwarp();  // orders the leader's acquire before the group's gathers
            got = __shfl_sync(0xffffffffu, got, lane & ~(G - 1));
            if (act && !got) {
                act = false;
                len = 0;
                if (sl == 0) ++skipped;
            }
        }
        XT acc = 0;
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const int off = (c * G + sl) * 4;
            if (off < len) acc += dot4(vv[c], cc[c], len - off, x);
        }
        for (int off = (CH * G + sl) * 4; off < len; off += 4 * G) {  // rows longer than 4*G*CH
            XT v4[4];
            const int4 c4 = ld_col4(a.col + start + off);
            ld_val4(val + start + off, v4);
            acc += dot4(v4, c4, len - off, x);
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);

        if (act) {
            XT s;
            if (F64) {
                s = -((gamma * (acc - b)) / scale);  // the oracle's (gamma r) / ||a_i||^2
            } else {
                s = -(gamma * (acc - b) * scale);
            }
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const int off = (c * G + sl) * 4;
                if (off < len) scatter4(vv[c], cc[c], len - off, s, x);
            }
            for (int off = (CH * G + sl) * 4; off < len; off += 4 * G) {
                XT v4[4];
                const int4 c4 = ld_col4(a.col + start + off);
                ld_val4(val + start + off, v4);
                scatter4(v4, c4, len - off, s, x);
            }
        }
        if (EXCL) {
            __syncwarp();  // the group's updates happen before the leader's release
            if (act && sl == 0) release_row(a.busy, i);
        }
        if (SEQ) {
            __threadfence();
            __syncwarp();
        }
    }
    if (EXCL && skipped) atomicAdd(a.skipped, skipped);
}

__global__ void k_draw_rows(const RowRec *__restrict__ rec, uint2 key, unsigned m, int uniform,
                            unsigned stream_id, unsigned long long j0, long long count,
                            int32_t *__restrict__ out)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    RowRec r;
    out[t] = (int32_t)draw_row(j0 + (unsigned long long)t, stream_id, key, m, uniform, rec, r);
}

// ---------------------------------------------------------------------------
// dispatch
// ---------------------------------------------------------------------------
using KernelFn = void (*)(const ProjArgs);

template <typename VT, typename XT, bool SEQ, bool EXCL>
static KernelFn pick_g(int G)
{
    switch (G) {
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
    KernelFn k = pick_kernel(p->dtype, L.x_f64, L.sequential, excl, L.subwarp);
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
    a.busy = p->busy;
    a.skipped = p->skipped;
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
                     unsigned stream_id, int32_t *rows_dev, cudaStream_t s)
{
    const uint2 key = make_uint2((unsigned)p->seed, (unsigned)(p->seed >> 32));
    const long long blocks = (count + 255) / 256;
    k_draw_rows<<<(unsigned)blocks, 256, 0, s>>>(p->rec, key, (unsigned)p->m, p->uniform,
                                                   stream_id, j0, count, rows_dev);
    ASYRK_CK(cudaGetLastError());
    return ASYRK_OK;
}

}  // namespace asyrk
