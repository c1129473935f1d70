// common.cuh -- internal types and device helpers of libasyrk.so.
//
// Device layout of a problem (all in HBM, written once by asyrk_create):
//   rec[m]        32-byte row records: padded start, length, alias threshold,
//                 alias row, b_i and 1/||a_i||^2 at FP32.  The alias entry of
//                 bucket i and row i's own data share one 32-byte sector, so a
//                 draw that keeps its bucket costs one sector read.
//   col[nnz_pad]  int32 column indices, each row starting at a multiple of 4
//                 entries (padding entries hold column 0 and value 0 and are
//                 never used), so a lane loads 4 columns with one 16-byte load.
//   val[nnz_pad]  values in the stored dtype, same padding.
//   b64[m], w64[m]  b_i and ||a_i||^2 in FP64 (FP64 iterate paths, residuals).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "asyrk.h"

#define ASYRK_MAX_RED_BLOCKS 1024

struct __align__(32) RowRec {
    long long start;  // first stored entry of the row (multiple of 4)
    unsigned len;     // ||a_i||_0
    unsigned thr;     // alias threshold of bucket i: keep i if u1 < thr
    unsigned alias;   // alias row of bucket i
    float b;          // b_i (or the refinement residual r_i) at FP32
    float inv;        // 1 / ||a_i||^2 at FP32
    unsigned pad;
};
static_assert(sizeof(RowRec) == 32, "row record must be one 32-byte sector");

// bfloat16 stored as its 16-bit pattern; widening to FP32 is exact.
struct bf16_t {
    unsigned short bits;
};

#include "handle.cuh"  // struct asyrk_problem: host-side state of a handle

namespace asyrk {

// ---------------------------------------------------------------------------
// error reporting
// ---------------------------------------------------------------------------
int set_error(int status, const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what, const char *file, int line);

#define ASYRK_CK(call)                                                      \
    do {                                                                    \
        cudaError_t e__ = (call);                                           \
        if (e__ != cudaSuccess) return ::asyrk::cuda_fail(e__, #call, __FILE__, __LINE__); \
    } while (0)

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32
// multiplies whose high and low halves are mixed with the other two counter
// words and the key; the key is bumped by two Weyl constants between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
    const unsigned M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const unsigned W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        const unsigned hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += W0;
        k.y += W1;
    }
    return c;
}

__device__ __forceinline__ RowRec load_rec(const RowRec *p)
{
    const int4 *q = reinterpret_cast<const int4 *>(p);
    int4 a = __ldg(q), b = __ldg(q + 1);
    RowRec r;
    r.start = (long long)(((unsigned long long)(unsigned)a.y << 32) | (unsigned)a.x);
    r.len = (unsigned)a.z;
    r.thr = (unsigned)a.w;
    r.alias = (unsigned)b.x;
    r.b = __int_as_float(b.y);
    r.inv = __int_as_float(b.z);
    r.pad = (unsigned)b.w;
    return r;
}

// Row of projection j: Philox at counter (j_lo, j_hi, stream, 0), bucket =
// floor(u0 m / 2^32), keep the bucket when u1 < thr, else take its alias.
// Returns the row index and its record.
__device__ __forceinline__ unsigned draw_row(unsigned long long j, unsigned stream, uint2 key,
                                             unsigned m, int uniform, const RowRec *rec,
                                             RowRec &out)
{
    const uint4 u = philox4x32_10(make_uint4((unsigned)j, (unsigned)(j >> 32), stream, 0u), key);
    unsigned i = __umulhi(u.x, m);
    out = load_rec(rec + i);
    if (!uniform && u.y >= out.thr) {
        i = out.alias;
        out = load_rec(rec + i);
    }
    return i;
}

// ---------------------------------------------------------------------------
// Shuffled sweeps: projection j of sweep k = j div m, position q = j mod m,
// uses row pi_k(q), a bijection of [0, m): a 4-round balanced Feistel network
// on 2h bits (2^(2h) >= m, so at most 4m values) walked until it lands below m;
// round r xors into the left half the low h bits of MurmurHash3's 32-bit
// finalizer (Appleby) of (right half xor K_r), K_0..K_3 = Philox at counter
// (k_lo, k_hi, stream, 1).  After 4096 walks (never seen) q maps to itself.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned murmur_fmix32(unsigned h)
{
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

// half width h of the Feistel domain for m rows
static inline int shuffle_half_bits(long long m)
{
    int bits = 0;
    while ((1LL << bits) < m) ++bits;
    const int h = (bits + 1) / 2;
    return h < 1 ? 1 : h;
}

__device__ __forceinline__ unsigned shuffled_position(unsigned long long j, unsigned m,
                                                      unsigned stream, uint2 key, int h)
{
    const unsigned long long k = j / m;
    const unsigned q = (unsigned)(j - k * m);
    const uint4 K = philox4x32_10(make_uint4((unsigned)k, (unsigned)(k >> 32), stream, 1u), key);
    const unsigned mask = (h >= 32) ? 0xffffffffu : ((1u << h) - 1u);
    unsigned v = q;
    for (int walk = 0; walk < 4096; ++walk) {
        unsigned L = v >> h, R = v & mask, t;
        // four rounds, round r keyed by word r of K
        t = L ^ (murmur_fmix32(R ^ K.x) & mask); L = R; R = t;
        t = L ^ (murmur_fmix32(R ^ K.y) & mask); L = R; R = t;
        t = L ^ (murmur_fmix32(R ^ K.z) & mask); L = R; R = t;
        t = L ^ (murmur_fmix32(R ^ K.w) & mask); L = R; R = t;
        v = (L << h) | R;
        if (v < m) return v;
    }
    return q;
}

// ---------------------------------------------------------------------------
// launchers (defined in project.cu / measure.cu)
// ---------------------------------------------------------------------------
struct ProjectLaunch {
    asyrk_problem *p = nullptr;
    void *x = nullptr;              // float* or double*
    bool x_f64 = false;
    double gamma = 1.0;
    unsigned long long j0 = 0;
    unsigned long long count = 0;   // projections in this launch
    unsigned stream_id = 0;
    int workers = 1;                // concurrent row groups
    int subwarp = 32;               // lanes per row group
    bool sequential = false;        // one group, strictly ordered projections
    bool exclusive = true;          // row exclusion (skip rows another worker holds)
    int sampling = 0;               // 0: weighted i.i.d. draws, 1: shuffled sweeps
    int update = 0;                 // 0: the whole row, 1: one coordinate (Algorithm 1)
    bool b_from_rec = true;         // FP32 b from rec (else b64)
    const unsigned long long *dyn = nullptr;  // device {j0, count} (graph-captured loop)
    int form = 0;                   // 0: by warps per SM, 1: latency form, -1: throughput form
    cudaStream_t stream = nullptr;
};
int launch_project(const ProjectLaunch &L);  // counts into L.p->launches
int project_max_workers(const asyrk_problem *p, bool x_f64, int subwarp, int *max_workers);
int choose_subwarp(int64_t max_len, int64_t nnz, int64_t m);

int launch_draw_rows(const asyrk_problem *p, unsigned long long j0, int64_t count,
                     unsigned stream_id, int sampling, int32_t *rows_dev, cudaStream_t s);

// FP64 reductions; each leaves its result(s) in p->red_out[slot...]
int launch_err2(asyrk_problem *p, const void *x, bool x_f64, const double *xt, int slot,
                cudaStream_t s);
int launch_sumsq(asyrk_problem *p, const double *v, int64_t n, int slot, cudaStream_t s);
// ||A^T (A x - b)||^2 in FP64 into red_out[slot]
int launch_normal_residual(asyrk_problem *p, const void *x, bool x_f64, int slot, cudaStream_t s);
int launch_residual(asyrk_problem *p, const void *x, bool x_f64, bool write_rec_b, int slot,
                    cudaStream_t s);
int launch_convert(const void *src, bool src_f64, void *dst, bool dst_f64, int64_t n,
                   cudaStream_t s);
int launch_axpy_f32_to_f64(double *x64, const float *d, int64_t n, cudaStream_t s);
int launch_restore_rec_b(asyrk_problem *p, cudaStream_t s);

int ensure_workspace(asyrk_problem *p);

}  // namespace asyrk
