// cluster.cuh -- the on-chip batched solver (cluster.cu): one thread-block
// cluster per system, the system's FP32 iterate and row-claim bits held in the
// cluster's distributed shared memory for the whole solve.
#pragma once

#include "common.cuh"

namespace asyrk {

constexpr int CLUSTER_MAX_THREADS = 1024;          // threads per CTA
constexpr int CLUSTER_MAX_SIZE = 8;                // CTAs per cluster (portable limit)
// One CTA unless asked otherwise: measured on a GB300, a worker's projection
// takes ~2 us with the iterate in its own CTA's shared memory and 5.5-8.8 us
// when its gathers and updates go to other CTAs of a cluster of 2-8.
constexpr int CLUSTER_DEFAULT_MAX = 1;
constexpr size_t CLUSTER_SMEM_BYTES = 200 * 1024;  // dynamic shared memory per CTA, at most
constexpr int SERVER_ONCHIP_SLOTS = 64;            // on-chip requests a server runs at once
// Cost model of a hybrid batch (measured on a GB300): the time one worker
// takes per projection with the iterate in its CTA's shared memory (2.0 us
// on a system whose rows stay in L2, 2.6 us on the largest members of the
// batched workload, which stream theirs from HBM; the model takes the latter;
// rows
// whose chunks of 4 entries per lane fit the registers that hold them; each
// further chunk, loaded after them and re-read for the update, adds 45 %) and
// with the iterate in L2,
// and the projection rate of the global-iterate engine over the whole GPU
// (1.6-1.8 G/s on parts of the 256-system batched workload).
constexpr double ONCHIP_SECONDS_PER_PROJECTION = 2.6e-6;
constexpr double ONCHIP_TAIL_CHUNK_FACTOR = 0.45;
constexpr double GLOBAL_SECONDS_PER_PROJECTION = 4.5e-6;
constexpr double GLOBAL_PROJECTIONS_PER_SECOND = 1.7e9;
constexpr double THREADS_PER_SM = 2048.0;

// One solve, read by its cluster (a batch member or a served request); the
// host writes the per-solve fields before the launch and reads the results
// after it.
struct ClusterJob {
    const RowRec *rec;
    const int32_t *col;
    const void *val;
    double *x64;       // in: x0 (FP64); refinement: the FP64 iterate, in and out
    float *x32;        // out: x (FP32; plain solves)
    const double *xt;  // x* in FP64, or nullptr: measure ||b - A x|| / ||b||
    const double *b64; // FP64 b (refinement's outer residual)
    float *r32;        // refinement: workspace of m floats, r = b - A x64 at FP32
    uint2 key;
    unsigned m, n;
    unsigned stream_id;  // Philox stream of the row sequence (a served request's ticket)
    int uniform;
    int sampling;      // 0: weighted i.i.d. draws, 1: shuffled sweeps
    int shuf_h;
    int excl;          // row exclusion
    int workers;       // W (1: one worker, strictly sequential projections)
    int lc;            // log2 of the cluster size C
    int nper;          // x entries per CTA: ceil(n / C)
    int nper_pad;      // nper rounded up to 4 (the claim words follow)
    int bper;          // claim words per CTA: ceil(ceil(m / 32) / C)
    float gamma;
    int refine;        // 1: FP64 iterate x64 refined by FP32 inner solves (d on chip)
    int pad0;
    long long max_inner;  // refinement: inner sweeps per outer step at most
    double inner_tol;     // refinement: inner target ||r - A d|| / ||r||
    // per solve
    unsigned long long j0;  // first projection of the row sequence
    long long max_sweeps;
    double tol;
    double bnorm;      // ||b|| (reference of the residual measure)
    // results
    double meas, meas0;
    long long sweeps;
    unsigned long long skipped;
    int status;
    int outer_steps;   // refinement: outer steps taken
    double res2;       // refinement: ||b - A x64||^2 of the last outer step
};

struct ClusterShape {
    int fits;        // 0: the system does not fit a cluster's shared memory
    int C, lc;       // CTAs per cluster and log2 C
    int threads;     // per CTA
    int workers;     // W
    int G;           // lanes per row
    size_t smem;     // dynamic shared memory per CTA
    int nper, nper_pad, bper;
};

// Shape of the cluster for problem p at sub-warp width G with at most
// cluster_max CTAs (0: the default) and max_workers workers (0: the Cor. 2
// estimate); sh->fits = 0 when it does not fit.
int cluster_shape(const asyrk_problem *p, int G, int cluster_max, int max_workers,
                  ClusterShape *sh);
// Allow the kernel for (dtype, G, C > 1) its shared memory (once per device).
int cluster_prepare(int dtype, int G, int C);
// EINVAL when a cluster of this shape can never be resident on the device.
int cluster_check_schedulable(int dtype, const ClusterShape &sh);
// The solve of jobs[k] as a kernel node of g (no dependencies).
int cluster_add_node(cudaGraph_t g, int dtype, const ClusterShape &sh, ClusterJob *jobs, int k);
// One kernel node of g solving several one-CTA members: CTA b solves
// jobs[list[b]] (list: `ctas` device ints), every CTA with `threads` threads and
// `smem` bytes of dynamic shared memory (at least each member's own).
int cluster_add_list_node(cudaGraph_t g, int dtype, int G, int threads, size_t smem, int ctas,
                          ClusterJob *jobs, const int *list);
// The solve of jobs[k] launched on s.
int cluster_launch(int dtype, const ClusterShape &sh, ClusterJob *jobs, int k, cudaStream_t s);

}  // namespace asyrk
