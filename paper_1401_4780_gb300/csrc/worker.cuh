// worker.cuh -- the per-projection work of one row worker, shared by the
// single-system kernel (project.cu) and the multi-system kernel (batch.cu).
//
// One "worker" is a group of G lanes of a warp (G = 2..32), so a warp runs
// 32/G workers side by side.  For each projection (Section 3's five
// per-thread steps, with the full-row update of Section 5):
//   1. draw the row i (Philox counter j, alias table; one 32-byte record);
//   2. load the row's columns and values, 4 per lane with 16-byte loads;
//   3. gather x on supp(a_i) from L2 and reduce a_i^T x across the G lanes;
//   4. s = -gamma (a_i^T x - b_i) / ||a_i||^2;
//   5. x_t += s * A_it for every t in supp(a_i), each as one red.global.add
//      (an atomic add that returns nothing; no locks, Section 3).
// Reads of x are not synchronised with other workers' updates, so a worker
// may project with an x that misses up to about W - 1 concurrent updates:
// the staleness bound tau of Eq. (4) is set by W.
#pragma once

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
    const float *bvec;               // FP32 right-hand side replacing rec.b, or nullptr
    int sampling;                    // 0: weighted i.i.d. draws, 1: shuffled sweeps
    int shuf_h;                      // half width of the shuffle's Feistel domain
    int update;                      // 0: the whole row, 1: one coordinate (Algorithm 1)
    unsigned *busy;                  // row-claim bits (row exclusion)
    unsigned long long *skipped;     // projections skipped by row exclusion
    const unsigned long long *dyn;   // non-null: j0 = dyn[0], count = dyn[1] (device loop)
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

// one entry (the single-coordinate update)
__device__ __forceinline__ double ld_val1(const double *p) { return __ldcs(p); }
__device__ __forceinline__ float ld_val1(const float *p) { return __ldcs(p); }
__device__ __forceinline__ float ld_val1(const bf16_t *p)
{
    return __uint_as_float((unsigned)__ldcs(reinterpret_cast<const unsigned short *>(p)) << 16);
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
// L2) with an atomic OR before gathering x, and clears the bit after issuing
// its updates; a row whose bit is already set is skipped.  So no row is held
// by two workers at once -- many copies of one (heavily weighted) row would
// apply the same correction again and again from the same stale x -- the
// property the paper's implementation gets from giving each thread its own
// rows (Section 5).  The skipped projection would, in the sequential order,
// come right after the same projection and change x only through the few
// updates in between (projections are idempotent).
// Both operations are relaxed: the next holder may still read x before the
// previous holder's red.adds have landed, the same bounded staleness every
// read of x has.  Release ordering would make the clearing lane wait for all
// of its outstanding red.adds, which costs about a fifth of the throughput.
__device__ __forceinline__ unsigned claim_row(unsigned *busy, unsigned i)
{
    unsigned old;
    asm volatile("atom.relaxed.gpu.global.or.b32 %0, [%1], %2;"
                 : "=r"(old)
                 : "l"(busy + (i >> 5)), "r"(1u << (i & 31))
                 : "memory");
    return !(old & (1u << (i & 31)));
}

__device__ __forceinline__ void release_row(unsigned *busy, unsigned i)
{
    asm volatile("red.relaxed.gpu.global.and.b32 [%0], %1;" ::"l"(busy + (i >> 5)),
                 "r"(~(1u << (i & 31)))
                 : "memory");
}

template <typename VT, typename XT, int G, bool SEQ, bool EXCL, bool DYN = true>
__device__ __forceinline__ unsigned long long run_workers(const ProjArgs &a, long long gbase,
                                                          long long W)
{
    constexpr int CH = 1;        // row chunks of 4G entries kept in registers (longer rows
                                 // re-read their tail for the scatter)
    constexpr bool F64 = std::is_same<XT, double>::value;
    const int lane = threadIdx.x & 31;
    const int sub = lane / G, sl = lane % G;
    if (gbase >= W) return 0;  // whole warp idle
    const bool worker = gbase + sub < W;
    const VT *__restrict__ val = static_cast<const VT *>(a.val);
    XT *x = static_cast<XT *>(a.x);
    const XT gamma = (XT)a.gamma;
    unsigned long long skipped = 0;

    // the launch's position and length: arguments, or device words that a
    // graph-captured loop advances between launches
    unsigned long long dj0 = 0, dcount = 0;
    if (DYN) {
        dj0 = a.dyn ? __ldcg(a.dyn) : a.j0;
        dcount = a.dyn ? __ldcg(a.dyn + 1) : a.count;
    }
#define ASYRK_J0 (DYN ? dj0 : a.j0)
#define ASYRK_COUNT (DYN ? dcount : a.count)

    // t0 walks k*W + gbase, so worker gbase+sub gets projection t0 + sub.  The
    // trip count is warp-uniform: every lane reaches every shuffle and barrier.
    for (unsigned long long t0 = (unsigned long long)gbase; t0 < ASYRK_COUNT;
         t0 += (unsigned long long)W) {
        const unsigned long long t = t0 + sub;
        bool act = worker && t < ASYRK_COUNT;
        long long start = 0;
        int len = 0;
        unsigned i = 0, pick = 0;
        XT b = 0, scale = 0;
        if (act) {
            RowRec r;
            const unsigned long long j = ASYRK_J0 + t;
            if (a.sampling == 1) {
                i = shuffled_position(j, a.m, a.stream_id, a.key, a.shuf_h);
                r = load_rec(a.rec + i);
            } else {
                i = draw_row(j, a.stream_id, a.key, a.m, a.uniform, a.rec, r);
            }
            start = r.start;
            len = (int)r.len;
            if (a.update == 1) {  // the entry of Algorithm 1: u2 of projection j
                const uint4 u = philox4x32_10(
                    make_uint4((unsigned)j, (unsigned)(j >> 32), a.stream_id, 0u), a.key);
                pick = __umulhi(u.z, (unsigned)len);
            }
            if (F64) {
                b = (XT)__ldg(a.b64 + i);
                scale = (XT)__ldg(a.w64 + i);
            } else {
                b = a.bvec ? (XT)__ldg(a.bvec + i) : (XT)r.b;
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

        if (act && a.update == 1) {
            // one coordinate: x_t -= gamma theta_i A_it r / ||a_i||^2
            XT s;
            if (F64) {
                s = -((gamma * (acc - b)) / scale);
            } else {
                s = -(gamma * (acc - b) * scale);
            }
            if (sl == 0) {
                const long long k = start + pick;
                red_add(x + a.col[k], ((XT)len * s) * (XT)ld_val1(val + k));
            }
        } else if (act) {
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
            __syncwarp();  // the group's updates are issued before the bit is cleared
            if (act && sl == 0) release_row(a.busy, i);
        }
        if (SEQ) {
            __threadfence();
            __syncwarp();
        }
    }
    return skipped;
#undef ASYRK_J0
#undef ASYRK_COUNT
}

// ---------------------------------------------------------------------------
// The latency form of run_workers, for launches with a few warps per SM (small
// systems, whose worker count Corollary 2 caps near m / (2e lambda_max)).  There
// a worker's projections follow one another with nothing to hide their round
// trips to L2: the row record, the row, then the gathers.  Here a worker draws
// its record two projections ahead and loads its row (and, with FP64 values,
// b_i and ||a_i||^2) one ahead, and sends a projection's claim and gathers out
// together with those loads, so that a projection waits about one round trip.
// The projections, their order per worker and the number in flight (the delay
// tau) are those of run_workers; the gathers of a projection whose claim fails
// are dropped unused.  Full-row updates, i.i.d. or shuffled draws.
// ---------------------------------------------------------------------------
using ProjKernelFn = void (*)(const ProjArgs);
// the latency form of the projection kernel (project_pf.cu); nullptr for an unknown G
ProjKernelFn pick_project_pf(int dtype, bool x_f64, bool excl, int G);

template <typename XT>
struct Ahead {
    long long start;
    int len;  // 0: no projection (past the launch, or a lane without a worker)
    unsigned i;
    XT b, scale;
    int4 cc;     // this lane's first 4-entry chunk of the row
    XT vv[4];
};

// the record of projection t of the launch
template <typename XT>
__device__ __forceinline__ void pf_draw(const ProjArgs &a, bool worker, unsigned long long j0,
                                        unsigned long long count, unsigned long long t, Ahead<XT> &q)
{
    constexpr bool F64 = std::is_same<XT, double>::value;
    q.len = 0;
    q.start = 0;
    q.i = 0;
    q.b = 0;
    q.scale = 0;
    if (!worker || t >= count) return;
    RowRec r;
    const unsigned long long j = j0 + t;
    if (a.sampling == 1) {
        q.i = shuffled_position(j, a.m, a.stream_id, a.key, a.shuf_h);
        r = load_rec(a.rec + q.i);
    } else {
        q.i = draw_row(j, a.stream_id, a.key, a.m, a.uniform, a.rec, r);
    }
    q.start = r.start;
    q.len = (int)r.len;
    if (!F64) {
        q.b = a.bvec ? (XT)__ldg(a.bvec + q.i) : (XT)r.b;
        q.scale = (XT)r.inv;
    }
}

// the loads of projection q that need its record: the lane's chunk of the row,
// and b_i and ||a_i||^2 in FP64
template <typename VT, typename XT>
__device__ __forceinline__ void pf_fetch(const ProjArgs &a, const VT *val, int off, Ahead<XT> &q)
{
    constexpr bool F64 = std::is_same<XT, double>::value;
    if (off < q.len) {
        q.cc = ld_col4(a.col + q.start + off);
        ld_val4(val + q.start + off, q.vv);
    }
    if (F64 && q.len > 0) {
        q.b = (XT)__ldg(a.b64 + q.i);
        q.scale = (XT)__ldg(a.w64 + q.i);
    }
}

// Projection cur (record and chunk loaded ahead); meanwhile the row of nxt is
// loaded and the record of the projection after nxt (t_after) is drawn into
// cur's slot.
template <typename VT, typename XT, int G, bool EXCL>
__device__ __forceinline__ void pf_step(const ProjArgs &a, const VT *val, XT *x, XT gamma,
                                        int lane, int sl, bool worker, unsigned long long j0,
                                        unsigned long long count, unsigned long long t_after,
                                        Ahead<XT> &cur, Ahead<XT> &nxt,
                                        unsigned long long &skipped)
{
    constexpr bool F64 = std::is_same<XT, double>::value;
    const int off = sl * 4;
    bool act = cur.len > 0;
    unsigned got = 1;
    if (EXCL && act && sl == 0) got = claim_row(a.busy, cur.i);
    const int k = cur.len - off;  // entries of the row in this lane's first chunk
    XT xv[4] = {0, 0, 0, 0};
    if (k > 0) {
        xv[0] = ld_x(x + cur.cc.x);
        if (k > 1) xv[1] = ld_x(x + cur.cc.y);
        if (k > 2) xv[2] = ld_x(x + cur.cc.z);
        if (k > 3) xv[3] = ld_x(x + cur.cc.w);
    }
    pf_fetch<VT, XT>(a, val, off, nxt);
    Ahead<XT> nn;
    pf_draw<XT>(a, worker, j0, count, t_after, nn);
    if (EXCL) {
        got = __shfl_sync(0xffffffffu, got, lane & ~(G - 1));
        if (act && !got) {
            act = false;
            if (sl == 0) ++skipped;
        }
    }
    XT acc = 0;
    if (act && k > 0) {  // the order of dot4
        acc = cur.vv[0] * xv[0];
        if (k > 1) acc += cur.vv[1] * xv[1];
        if (k > 2) acc += cur.vv[2] * xv[2];
        if (k > 3) acc += cur.vv[3] * xv[3];
    }
    if (act) {
        for (int o = (G + sl) * 4; o < cur.len; o += 4 * G) {  // rows longer than 4*G
            XT v4[4];
            const int4 c4 = ld_col4(a.col + cur.start + o);
            ld_val4(val + cur.start + o, v4);
            acc += dot4(v4, c4, cur.len - o, x);
        }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (act) {
        XT s;
        if (F64) {
            s = -((gamma * (acc - cur.b)) / cur.scale);
        } else {
            s = -(gamma * (acc - cur.b) * cur.scale);
        }
        if (k > 0) scatter4(cur.vv, cur.cc, k, s, x);
        for (int o = (G + sl) * 4; o < cur.len; o += 4 * G) {
            XT v4[4];
            const int4 c4 = ld_col4(a.col + cur.start + o);
            ld_val4(val + cur.start + o, v4);
            scatter4(v4, c4, cur.len - o, s, x);
        }
    }
    if (EXCL) {
        __syncwarp();  // the group's updates are issued before the bit is cleared
        if (act && sl == 0) release_row(a.busy, cur.i);
    }
    cur.start = nn.start;
    cur.len = nn.len;
    cur.i = nn.i;
    cur.b = nn.b;
    cur.scale = nn.scale;
}

template <typename VT, typename XT, int G, bool EXCL, bool DYN = true>
__device__ __forceinline__ unsigned long long run_workers_pf(const ProjArgs &a, long long gbase,
                                                             long long W)
{
    const int lane = threadIdx.x & 31;
    const int sub = lane / G, sl = lane % G;
    if (gbase >= W) return 0;  // whole warp idle
    const bool worker = gbase + sub < W;
    const VT *__restrict__ val = static_cast<const VT *>(a.val);
    XT *x = static_cast<XT *>(a.x);
    const XT gamma = (XT)a.gamma;
    unsigned long long skipped = 0;
    unsigned long long j0 = a.j0, count = a.count;
    if (DYN && a.dyn) {
        j0 = __ldcg(a.dyn);
        count = __ldcg(a.dyn + 1);
    }
    const unsigned long long w = (unsigned long long)W;
    // worker gbase+sub applies projections t = gbase + sub + k W; the two slots
    // take turns as the current projection and the next, so that a row's loads
    // stay in the registers they were issued to until it is worked on
    unsigned long long t = (unsigned long long)(gbase + sub);
    Ahead<XT> p0, p1;
    pf_draw<XT>(a, worker, j0, count, t, p0);
    pf_fetch<VT, XT>(a, val, sl * 4, p0);
    pf_draw<XT>(a, worker, j0, count, t + w, p1);
    // t0 = gbase + k W is warp-uniform: every lane reaches every shuffle and barrier
    for (unsigned long long t0 = (unsigned long long)gbase; t0 < count; t0 += 2 * w, t += 2 * w) {
        pf_step<VT, XT, G, EXCL>(a, val, x, gamma, lane, sl, worker, j0, count, t + 2 * w, p0, p1,
                                 skipped);
        if (t0 + w >= count) break;
        pf_step<VT, XT, G, EXCL>(a, val, x, gamma, lane, sl, worker, j0, count, t + 3 * w, p1, p0,
                                 skipped);
    }
    return skipped;
}

}  // namespace asyrk
