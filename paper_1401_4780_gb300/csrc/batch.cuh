// batch.cuh -- many independent systems ("slots") advanced by one persistent
// projection kernel, shared by the batched solve (batch.cu) and the server
// (server.cu).
//
// One iteration of the engine is four kernels:
//   plan     split the resident warps among the active slots in proportion to
//            their work per sweep, each capped by its concurrency limit (the
//            tau bound of Cor. 2, expressed in warps), and let a slot whose
//            sweep is short next to the step's longest run up to max_k sweeps;
//   project  every warp finds its slot and runs that slot's workers for its
//            k sweeps (k m_s projections) with the slot's value type and
//            sub-warp width (worker.cuh);
//   check    the slot's FP64 error measure (||x - x*|| / ||x*|| with x*, else
//            ||b - A x|| / ||b||), its sweep count and done/status;
//   cond     count the active slots; in a CUDA graph, set the WHILE condition.
#pragma once

#include "common.cuh"

namespace asyrk {

constexpr int BATCH_ERR_CHUNK = 16384;  // x entries per check block (x* measure)
constexpr int BATCH_ROW_CHUNK = 2048;   // rows per check block (residual measure)
constexpr int BATCH_MAX_SLOTS = 4096;   // slots the plan kernel can place
// projections per worker a server step runs at least (a lone large request of
// the served workload sweeps in ~50 per worker), capped per slot by the
// sweeps its measured contraction says it still needs; only the server's steps
constexpr double SERVER_STEP_CHAIN = 512.0;

struct SysDesc {
    const RowRec *rec;
    const int32_t *col;
    const void *val;
    const double *b64;  // FP64 b of the problem (final residual)
    const float *bvec;  // FP32 right-hand side replacing rec.b, or nullptr
    float *x;           // FP32 iterate of this slot
    double *x64;        // FP64 staging of this slot's x (in/out)
    const double *xt;   // x* in FP64, or nullptr: residual measure
    unsigned *busy;     // row-claim bits of this slot
    double ref;         // ||x*|| or ||b||; < 0: computed by the first check
    double tol;
    double meas;        // last check measure
    double meas0;       // first measure (divergence test)
    double res2, bb2;   // final FP64 ||b - A x||^2 and ||b||^2
    double work;        // stored entries per sweep
    unsigned long long j;        // next projection of the slot's row sequence
    unsigned long long skipped;  // projections skipped by row exclusion
    long long sweeps;
    long long max_sweeps;
    uint2 key;
    unsigned m, n;
    unsigned stream_id;
    float gamma;
    int dtype;
    int G;
    int cap_warps;  // concurrency cap in warps
    int uniform;
    int active;     // 1 while being solved
    int status;
    int warp0, nwarps;    // this iteration's warps
    int first_nwarps;     // warps of the first iteration (reported)
    int chunk0, nchunks;  // check blocks of this slot
    unsigned chk_count;   // last-block counter of the check
    unsigned res_count;   // last-block counter of the final residual
    // mixed-precision refinement (mode 1): x is the FP32 correction d, x64 the
    // FP64 iterate, r32 the FP32 right-hand side r = b - A x64 of the inner solve
    int mode;             // 0: plain FP32 solve, 1: FP64 refinement
    int phase;            // 0: projections; 1: outer step pending
    float *r32;
    double inner_tol;     // inner solve: ||r - A d|| / ||r|| target
    double inner_goal;    // this outer step's inner target: inner_tol, or the
                          // reduction the tolerance still needs when closer
    long long inner_sweeps, max_inner;
    int outer_steps;
    unsigned out_count;   // last-block counter of the outer step
    double outer_ref;     // ||x*|| (with x*) or ||b|| for the outer measure
    int max_k;            // sweeps one engine step may run for this slot (>= 1)
    int k;                // sweeps this step (set by plan)
    int sampling;         // 0: weighted i.i.d. draws, 1: shuffled sweeps
    int update;           // 0: the whole row, 1: one coordinate (Algorithm 1)
    int shuf_h;           // half width of the shuffle's Feistel domain
    int pad2;
};
// The inner target of an outer refinement step: inner_tol, or, when the outer
// measure `meas` is within a factor 1/inner_tol of the tolerance, half the
// reduction it still needs (at most 1/2), so the last inner solve stops near
// the tolerance instead of far below it.
__host__ __device__ __forceinline__ double refine_inner_goal(double inner_tol, double tol,
                                                             double meas)
{
    if (!(tol > 0.0) || !(meas > 0.0)) return inner_tol;
    const double need = 0.5 * tol / meas;
    return need > inner_tol ? (need < 0.5 ? need : 0.5) : inner_tol;
}


constexpr int SLOT_PLAIN = 0;
constexpr int SLOT_REFINE = 1;

// warps of the project kernel that are resident on the whole GPU at once
int batch_resident_warps(int sm_count, bool excl, int *warps);

// One engine iteration (plan, project, check, cond) enqueued on s.  d_iter[0]
// counts iterations, d_iter[1] bounds them; d_active receives the active slots.
// use_cond: call cudaGraphSetConditional(h, ...) (only inside a graph).
int launch_batch_iteration(SysDesc *d, int count, int total_chunks, double *part,
                           int resident_warps, bool excl, int *d_active, int *d_iter,
                           bool use_cond, unsigned long long cond_handle, cudaStream_t s);

// The check alone with measure_only: first measure (and ||x*||), no sweep.
int launch_batch_measure(SysDesc *d, int count, int total_chunks, double *part, cudaStream_t s);

// Final FP64 residual of every slot from its x64 staging (res2, bb2).
int launch_batch_residual(SysDesc *d, int count, int total_chunks, double *part, cudaStream_t s);

// plan, project, check and (with_outer) the outer step of refinement slots
// whose phase is 1: x64 += d, d = 0, then r = b - A x64 in FP64 (stored to
// r32), the outer measure and the decision.  Returns without a cond kernel.
int launch_engine_step(SysDesc *d, int count, int total_chunks, double *part, int resident_warps,
                       bool excl, bool with_outer, cudaStream_t s);
int launch_batch_outer(SysDesc *d, int count, int total_chunks, double *part, cudaStream_t s);

int choose_subwarp(int64_t max_len, int64_t nnz, int64_t m);
int tuned_subwarp(int dtype, int64_t max_len, int64_t nnz, int64_t m, bool *found);

// Sub-warp width of a slot in the multi-system engine: the single-system width
// (tuned, else the default); in a batched solve, half of it (at least one lane).
// What counts for a batch is its total time, and a slot's share of the GPU leaves its
// workers latency-bound, so twice the rows per warp in flight pay (256-system
// batch: 92 ms against 97.5 ms at the full width, 94 ms at a quarter).  For a served
// solve it is the latency, and an engine step lasts as long as its
// longest worker chain, which the narrower width lengthens (p50 12 ms against
// 22 ms at Poisson 1000/s with the half width).
int engine_subwarp(const asyrk_problem *p, bool batched);
// x64 <-> x conversions over all slots (n_total entries laid out slot by slot)
int launch_batch_convert(const double *x64, float *x, int64_t n_total, bool to_f32, cudaStream_t s);

long long tau_cap_estimate(int64_t m, int64_t n);

// autotuned (sub-warp width, fraction of the resident workers) for problems of
// this value dtype and row-length class on this GPU, if asyrk_autotune ran
bool tuned_shape(int dtype, int64_t max_len, int *G, double *frac);

}  // namespace asyrk
