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
    constexpr int GPW = 32 / G;  // workers per warp
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

}  // namespace asyrk
