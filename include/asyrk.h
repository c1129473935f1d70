/*
 * asyrk.h -- C ABI of libasyrk.so: asynchronous parallel randomized Kaczmarz
 * (AsyRK; Liu, Wright, Sridhar, arXiv:1401.4780) on one NVIDIA GB300 GPU.
 *
 * The method solves a consistent sparse system A x = b (m x n, no zero rows;
 * Section 1 of the paper).  Many workers on the GPU repeatedly draw a row i
 * with probability ||a_i||^2 / ||A||_F^2 (Section 1, before Eq. (2)), read the
 * entries of a shared iterate x on supp(a_i), form r = a_i^T x - b_i and
 * apply the projection of Eq. (2) with a step-length factor gamma,
 *     x_t <- x_t - gamma * r * A_it / ||a_i||^2   for every t in supp(a_i),
 * to the shared x without locks (the full-row variant of Section 5; the
 * lock-free shared-memory model of Section 3, where the age of the x a worker
 * read is bounded by tau, Eq. (4), roughly the number of workers in flight).
 *
 * Conventions for every function below:
 *   - Return value: ASYRK_OK (0) on success; a negative asyrk_status is a
 *     hard error and leaves outputs unspecified; a positive status
 *     (NOT_CONVERGED, DIVERGED) is a solver outcome with outputs filled in.
 *     asyrk_last_error() gives a one-line description of the last hard error
 *     raised on the calling thread.
 *   - Pointers are host pointers unless the options say "device"; device
 *     pointers must be CUDA global memory of the current device.
 *   - The caller keeps ownership of every array it passes; the library
 *     copies what it needs.  A handle owns its device memory until destroyed.
 *   - All device work of a call is enqueued on the stream given in the
 *     options (NULL: the legacy default stream); a call returns after that
 *     stream has finished the call's work.
 *   - Handles are not thread-safe: one thread at a time per handle.
 *   - Row exclusion (ASYNC/REFINE, on by default): a worker claims its row
 *     before reading x and skips the projection if another worker holds the
 *     row, so no row is applied twice from the same stale x -- the property
 *     the paper's implementation gets from giving each thread its own rows
 *     (Section 5).  Skipped projections still advance the row sequence.
 *   - Row sampling is reproducible: projection number j of a problem draws
 *     its row from Philox4x32-10 (Salmon et al., SC'11) with key = seed and
 *     counter = (j mod 2^32, j div 2^32, stream id, 0): bucket =
 *     floor(u0 * m / 2^32); row = bucket if u1 < thr[bucket] else
 *     alias[bucket], where (thr, alias) is the alias table (Walker's method)
 *     of the row weights w_i = ||a_i||^2 (unused when all weights are
 *     bit-identical), built on the GPU and defined by one sweep:
 *     F = ||A||_F^2 is the exact sum of the w_i rounded once to the nearest
 *     double, ties to even (so it does not depend on any order of
 *     summation); integer masses M_i = floor(((w_i m) / F) 2^32)
 *     (one bucket is U = 2^32 units), the D = m U - sum M_i units lost to the
 *     floors added one per row from row 0 on (D / m to every row first when
 *     D >= m), an overshoot (D < 0) taken off the first row of largest mass;
 *     lights (M < U) and heavies (M >= U) each in index order; every light l
 *     in turn gets thr = M_l and alias = the heavy being drawn down, whose
 *     residual drops by U - M_l; while that residual R is below U the heavy
 *     gets thr = R, alias = the next heavy, and the next heavy's residual is
 *     its mass minus (U - R); the last heavy and heavies never drawn below U
 *     keep thr = 2^32 - 1 and alias = themselves.
 */
#ifndef ASYRK_H
#define ASYRK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ASYRK_ABI_VERSION 1

typedef struct asyrk_problem asyrk_problem; /* opaque; owns device copies of A, b, tables */

typedef enum asyrk_dtype {
    ASYRK_F64 = 0,  /* double values                                  */
    ASYRK_F32 = 1,  /* float values                                   */
    ASYRK_BF16 = 2  /* bfloat16 values given as uint16 bit patterns   */
} asyrk_dtype;

typedef enum asyrk_status {
    ASYRK_OK = 0,
    ASYRK_EINVAL = -1,        /* bad argument or malformed problem          */
    ASYRK_ENOMEM = -2,        /* device or host allocation failed           */
    ASYRK_ECUDA = -3,         /* a CUDA call failed                         */
    ASYRK_ETIMEOUT = -4,      /* a bounded wait gave up                     */
    ASYRK_ECANCELED = -5,     /* a served request was cancelled             */
    ASYRK_NOT_CONVERGED = 1,  /* max_sweeps reached above the tolerance     */
    ASYRK_DIVERGED = 2        /* the error measure became non-finite/huge   */
} asyrk_status;

typedef enum asyrk_mode {
    /* One worker (one warp), FP64 iterate, projections applied strictly in
     * order j = j0, j0+1, ...: the sequential RK iterate of Eq. (2), which is
     * what the paper's scheme is on a single thread (Section 5). */
    ASYRK_MODE_SEQUENTIAL = 0,
    /* Many lock-free workers updating x with atomic adds (Section 3): x is
     * FP64 for FP64 problems and FP32 otherwise. */
    ASYRK_MODE_ASYNC = 1,
    /* Mixed-precision iterative refinement (not in the paper): an FP64
     * iterate x64; each outer step computes r = b - A x64 in FP64 on the GPU,
     * solves A d = r with the ASYNC FP32 kernel and adds d to x64. */
    ASYRK_MODE_REFINE = 2
} asyrk_mode;

typedef enum asyrk_measure {
    /* ||x - x*|| / ||x*|| when x_true is given, else ||b - A x|| / ||b||  */
    ASYRK_MEASURE_AUTO = 0,
    /* ||b - A x|| / ||b|| (Section 5's figures plot ||Ax - b||)          */
    ASYRK_MEASURE_RESIDUAL = 1,
    /* ||A^T (A x - b)||^2, absolute (the measure of Table 2)            */
    ASYRK_MEASURE_NORMAL_RESIDUAL = 2
} asyrk_measure;

typedef enum asyrk_sampling {
    /* rows drawn i.i.d. with probability ||a_i||^2/||A||_F^2 (Section 1;
     * the analysis of Section 3): Philox and the alias table, as above      */
    ASYRK_SAMPLE_WEIGHTED = 0,
    /* every sweep of m projections visits each row once, in a new order per
     * sweep (the paper's implementation samples without replacement,
     * reshuffled after each scan, Section 5); row weights are not used.
     * Projection j of sweep k = j div m, position q = j mod m, uses row
     * pi_k(q): a 4-round balanced Feistel network on 2h bits (2^(2h) >= m)
     * walked until it lands below m, round r xoring into the left half the
     * low h bits of MurmurHash3's 32-bit finalizer of (right half xor K_r),
     * K_0..K_3 = Philox at counter (k_lo, k_hi, stream, 1)                   */
    ASYRK_SAMPLE_SHUFFLED = 1
} asyrk_sampling;

typedef enum asyrk_update {
    /* all of supp(a_i) (Section 5's implementation; Eq. (2))                */
    ASYRK_UPDATE_ROW = 0,
    /* one coordinate t, x_t -= gamma theta_i A_it r / ||a_i||^2, theta_i =
     * ||a_i||_0, t = floor(u2 theta_i / 2^32) with u2 the third Philox word of
     * the projection (Algorithm 1; with unit rows exactly its step)         */
    ASYRK_UPDATE_SINGLE = 1
} asyrk_update;

typedef struct asyrk_create_opts {
    uint64_t seed;       /* Philox key of the row sequence                       */
    int32_t device_ptrs; /* 1: row_ptr, col_idx, values, b are device pointers  */
    int32_t reserved;    /* must be 0                                            */
    void *stream;        /* cudaStream_t for the set-up work; NULL = default     */
} asyrk_create_opts;

typedef struct asyrk_solve_opts {
    int32_t mode;            /* asyrk_mode                                           */
    int32_t device_ptrs;     /* 1: x and x_true are device pointers (double)         */
    int32_t workers;         /* concurrent row workers; 0 = automatic (ASYNC/REFINE)  */
    int32_t subwarp;         /* lanes per row: 0 = automatic, or 1, 2, 4, 8, 16, 32   */
    int64_t check_every;     /* sweeps between convergence checks (>= 1); 0: adaptive,
                                half the sweeps the measured contraction still needs,
                                from 1 up to twice the last interval and a tenth of
                                the sweeps done (SEQUENTIAL and ASYNC; REFINE checks
                                every outer step)                                    */
    const double *x_true;    /* optional x*; checks then use ||x-x*||/||x*||          */
    void *stream;            /* cudaStream_t; NULL = legacy default stream           */
    double inner_tol;        /* REFINE: inner solve's target relative decrease (0: 1e-3) */
    int64_t inner_sweeps;    /* REFINE: inner sweeps per outer step (0: automatic)   */
    int32_t profile;         /* 1: time each projection launch with CUDA events      */
    int32_t row_exclusion;   /* ASYNC/REFINE: 0 or 1 = a worker skips a row that another
                                worker is applying (default); -1 = plain lock-free
                                updates, where one row may be applied several times
                                from the same stale x                                 */
    int32_t measure;         /* asyrk_measure of the convergence check               */
    int32_t sampling;        /* asyrk_sampling of the row sequence                   */
    int32_t update;          /* asyrk_update                                         */
    int32_t graph_loop;      /* 1: SEQUENTIAL/ASYNC solves with weighted sampling and
                                profile = 0 run their sweep-check loop inside one
                                CUDA graph (a WHILE node; the host waits once per
                                solve); 0 (default): the host drives the loop, one
                                wait per check                                      */
    int32_t kernel_form;     /* ASYNC/REFINE full-row projections: 0 (default) picks
                                the latency form -- each worker loads its next
                                projections' records and rows ahead -- for launches
                                of at most 8 warps per SM (small systems, whose
                                worker count Corollary 2 caps) and the throughput
                                form above; 1 always the latency form, -1 always
                                the throughput form.  Same projections, order per
                                worker and delay either way.  EINVAL: another
                                value, or 1 with UPDATE_SINGLE                       */
} asyrk_solve_opts;

typedef struct asyrk_solve_info {
    int32_t status;           /* same value as the return code                      */
    int32_t workers;          /* workers used (tau is about this many updates)      */
    int32_t subwarp;          /* lanes per row used                                 */
    int32_t refine_steps;     /* REFINE: outer steps taken                          */
    int64_t sweeps;           /* sweeps done (one sweep = m projections)            */
    int64_t projections;      /* projections done                                   */
    double seconds;           /* wall time of the call                              */
    double rel_err;           /* ||x-x*||/||x*|| at exit, or -1 without x_true      */
    double rel_res;           /* ||b-Ax||/||b|| at exit, FP64                       */
    double project_ms;        /* profile=1: summed event time of projection launches */
    int64_t project_launches; /* profile=1: number of projection launches timed      */
    uint64_t j_end;           /* position of the row sequence after the call        */
    int64_t kernel_launches;  /* GPU kernels this call launched (copies not counted) */
    int64_t skipped;          /* projections skipped by row exclusion (counted in
                                 `projections`)                                      */
} asyrk_solve_info;

typedef struct asyrk_problem_stats {
    int64_t m, n, nnz;        /* as created                                          */
    int64_t nnz_padded;       /* stored entries after padding rows to 4-aligned starts */
    int64_t max_row_len;      /* mu = max_i ||a_i||_0 (Section 1 notation)           */
    int64_t device_bytes;     /* device memory held by the handle                    */
    double frob2;             /* ||A||_F^2: the w_i's exact sum, rounded once        */
    int32_t dtype;            /* asyrk_dtype of the stored values                   */
    int32_t uniform;          /* 1: all row weights bit-identical, no alias table    */
    uint64_t seed;            /* Philox key                                          */
    uint64_t j_next;          /* next position of the row sequence                   */
} asyrk_problem_stats;

/* Create a problem from a CSR matrix A (m x n) and right-hand side b
 * (Section 1: A x = b consistent, no zero rows).
 *   row_ptr: m+1 int64, row_ptr[0] = 0, strictly increasing (no zero rows);
 *   col_idx: nnz int32, strictly ascending within each row, in [0, n);
 *   values : nnz entries of type vdtype (BF16 as uint16 bit patterns), finite,
 *            every row with ||a_i|| > 0;
 *   b      : m doubles, finite.
 * nnz = row_ptr[m]: col_idx and values must hold that many entries.  Host
 * arrays are read before the call returns (the entries in chunks on a stream
 * of the library's own, overlapping the checks and the row set-up); device
 * arrays too.
 * Errors: EINVAL (m, n outside [1, 2^31-1], a malformed CSR, a zero row,
 * non-finite data, ||A||_F^2 or ||b||^2 beyond the FP64 range, bad opts),
 * ENOMEM, ECUDA.  On error *out is NULL. */
int asyrk_create(asyrk_problem **out, int64_t m, int64_t n, const int64_t *row_ptr,
                 const int32_t *col_idx, const void *values, int vdtype, const double *b,
                 const asyrk_create_opts *opts);

/* Release the handle and its device memory (NULL is ignored). */
void asyrk_destroy(asyrk_problem *p);

/* Problems' device memory (arrays, set-up temporaries, solve workspace) comes
 * from one stream-ordered memory pool per device.  Memory that asyrk_destroy
 * frees stays in the pool, up to 1/8 of the device's memory and at most 16 GiB,
 * for the next asyrk_create on that device.  This call waits for the current
 * device and returns all the pool's unused memory to the driver.
 * Returns ASYRK_OK or ECUDA. */
int asyrk_trim_memory(void);

/* Run the method from x (in: x0, out: the final iterate; n doubles, host or
 * device per opts->device_ptrs) with step-length factor gamma in (0, 2)
 * (sequential RK contracts only there: the derivation before Eq. (3) gives a
 * decrease of gamma (2 - gamma) r^2/||a_i||^2 per step) until the check
 * measure is <= tol or max_sweeps sweeps are done.  The check measure, taken
 * every check_every sweeps in FP64 on the GPU, is ||x-x*||/||x*|| with
 * x_true, else ||b - A x||/||b|| (Section 5 plots ||Ax-b||).  tol <= 0 runs
 * exactly max_sweeps sweeps.  The row sequence continues from the problem's
 * position (asyrk_set_position) and the position advances by the
 * projections done.
 * Returns OK, NOT_CONVERGED, DIVERGED, or EINVAL (gamma outside (0, 2),
 * check_every < 0, max_sweeps < 0, mode or subwarp unknown, workers < 0),
 * ENOMEM, ECUDA.  info may be NULL. */
int asyrk_solve(asyrk_problem *p, double *x, double gamma, double tol, int64_t max_sweeps,
                const asyrk_solve_opts *opts, asyrk_solve_info *info);

/* ||b - A x||_2 / ||b||_2 in FP64 on the GPU (||b - A x|| when b = 0);
 * x: n doubles, host or device (x_on_device).  Errors: EINVAL, ECUDA. */
int asyrk_residual(asyrk_problem *p, const double *x, int x_on_device, double *rel_residual);

/* ||A^T (A x - b)||^2 in FP64 on the GPU (the measure of Table 2); x: n
 * doubles, host or device.  Errors: EINVAL, ENOMEM, ECUDA. */
int asyrk_normal_residual(asyrk_problem *p, const double *x, int x_on_device, double *value);

/* The rows drawn by projections j0 .. j0+count-1 with Philox stream id
 * `stream_id` under `sampling` (asyrk_sampling), computed by the GPU sampler
 * that the projection kernels use; rows_out: count int32 on the host.
 * Errors: EINVAL (count < 0, unknown sampling), ECUDA. */
int asyrk_draw_rows(asyrk_problem *p, uint64_t j0, int64_t count, uint32_t stream_id,
                    int sampling, int32_t *rows_out);

/* Position of the row sequence: the j of the next projection.  Saving it
 * with x and restoring both (asyrk_set_position) resumes a run; in
 * SEQUENTIAL mode the resumed run is identical to the uninterrupted one. */
int asyrk_get_position(asyrk_problem *p, uint64_t *j_next);
int asyrk_set_position(asyrk_problem *p, uint64_t j_next);

/* Sizes and statistics of a problem.  Errors: EINVAL. */
int asyrk_problem_get_stats(asyrk_problem *p, asyrk_problem_stats *stats);

/* ------------------------------------------------------------------------
 * Autotuner (not in the paper).  Times the projection kernel on problem p for
 * every sub-warp width (1..32 lanes per row) and for 1/2, 3/4 and all of the
 * resident workers (never above the Cor. 2 worker estimate m / (2 e
 * lambda_max) - 1 with lambda_max ~ (1 + sqrt(m/n))^2, Section 1), each for
 * `trial_projections` projections (0: min(2m, 2^22)) on a scratch iterate;
 * the problem's row-sequence position is not changed.  The fastest shape is
 * kept in a process-wide table keyed by (value dtype, row-length class =
 * max_row_len rounded up to a power of two, SM count) that asyrk_solve (with
 * subwarp = workers = 0) and asyrk_batch_create consult.  When the
 * environment variable ASYRK_TUNE_CACHE names a file, the table is read from
 * it on first use and rewritten after each tuning.
 * Errors: EINVAL, ECUDA, ENOMEM.
 * ------------------------------------------------------------------------ */
typedef struct asyrk_tune_result {
    int32_t subwarp;              /* chosen lanes per row                     */
    int32_t workers;              /* chosen concurrent workers                */
    double projections_per_s;     /* measured rate of the chosen shape        */
    int32_t trials;               /* shapes timed                             */
    int32_t from_cache;           /* 1: found in the table, nothing timed     */
} asyrk_tune_result;

int asyrk_autotune(asyrk_problem *p, int64_t trial_projections, int force, asyrk_tune_result *res);

/* ------------------------------------------------------------------------
 * Batched solves (not in the paper): many independent FP32/BF16 problems.
 * The global-iterate engine advances its members together by one persistent
 * projection kernel: each iteration splits the GPU's resident warps among the
 * unfinished problems in proportion to their stored entries, each capped by
 * its own Cor. 2 worker estimate, and runs one sweep of each; an FP64 check
 * then retires the problems that met their tolerance.  With graph >= 0 the
 * whole loop is one CUDA graph launch (a WHILE conditional node whose body is
 * that iteration; the device stops it), else a host loop.  The on-chip engine
 * (asyrk_engine below) takes the members that fit a CTA's shared memory.
 * ------------------------------------------------------------------------ */
typedef struct asyrk_batch asyrk_batch; /* opaque; owns per-problem iterates and tables */

/* Which engine advances a batch's members.  ONCHIP (not in the paper): a
 * member is solved by one CTA -- or a thread-block cluster of C <= cluster_max
 * CTAs -- that keeps its FP32 iterate and row-claim bits in shared memory for
 * the whole solve (gathers and atomic adds never leave the SM; only the row
 * stream comes from HBM), checks its measure after every sweep on the device
 * and writes x back at the end; such members run as independent nodes of one
 * CUDA graph.  It needs the full-row update and ceil(n/C) + ceil(m/32)/C
 * words per CTA within 200 KiB, and it gives a member at most the CTA's (or
 * cluster's) threads.  GLOBAL: the iterate-in-HBM/L2 engine described above,
 * which can give one member the whole GPU.  AUTO: the members that fit go
 * on-chip, except the largest ones while the global engine, running at the
 * same time on a second stream, would still finish first with them. */
typedef enum { ASYRK_ENGINE_AUTO = 0, ASYRK_ENGINE_GLOBAL = 1, ASYRK_ENGINE_ONCHIP = 2 } asyrk_engine;

typedef struct asyrk_batch_opts {
    void *stream;           /* cudaStream_t; NULL = legacy default stream          */
    int32_t graph;          /* >= 0: one graph launch per solve (default); -1: host loop
                               (ONCHIP: the members' launches one after another)   */
    int32_t row_exclusion;  /* as in asyrk_solve_opts                               */
    int32_t sampling;       /* asyrk_sampling of every member                       */
    int32_t update;         /* asyrk_update of every member                         */
    int32_t engine;         /* asyrk_engine (0: AUTO)                               */
    int32_t cluster_max;    /* ONCHIP: CTAs per cluster at most, 1, 2, 4 or 8 (0: 4) */
    int32_t workers;        /* ONCHIP: workers per member at most (0: the Cor. 2
                               estimate; 1: one worker, projections strictly in order) */
    int32_t partition;      /* both engines at once, graph form: >= 0 splits the SMs
                               between them, each engine on its own SMs, where the
                               driver offers SM partitions: 0 (default) sizes the
                               on-chip engine's share from its members' estimated
                               work, > 0 gives it that many SMs (kept within
                               [8, SMs - 8], rounded to the driver's granularity);
                               -1: both engines share every SM                      */
} asyrk_batch_opts;

typedef struct asyrk_batch_info {
    int32_t status;           /* OK if all converged, else the worst status        */
    int32_t converged;        /* problems that met their tolerance                 */
    int64_t iterations;       /* engine iterations (sweeps of the longest solve)   */
    int64_t projections;      /* projections over all problems                     */
    double seconds;           /* wall time of the call                             */
    double device_ms;         /* CUDA-event time of the iteration loop             */
    int64_t kernel_launches;  /* kernels run by the call (graph nodes included)    */
    int32_t resident_warps;   /* warps the engine splits among the problems        */
    int32_t graph;            /* 1: the loop ran as one graph launch               */
    int32_t engine;           /* engines that ran: GLOBAL (1), ONCHIP (2), both (3) */
    int32_t onchip_members;   /* members the on-chip engine solved                 */
    int32_t global_sms;       /* SMs of the global engine when the SMs were split
                                 between the engines, else 0                        */
    float global_ms;          /* CUDA-event time from the start of the loop to the
                                 end of the global engine's part (0: no members)   */
    float onchip_ms;          /* same, to the end of the on-chip engine's part     */
    int32_t reserved;
} asyrk_batch_info;

/* Group `count` problems (FP32 or BF16 values, all on the current device, each
 * at most once; count <= the resident warps, several thousand on a GB300).
 * The problems must outlive the batch.  Errors: EINVAL, ENOMEM, ECUDA. */
int asyrk_batch_create(asyrk_batch **out, asyrk_problem *const *problems, int count,
                       const asyrk_batch_opts *opts);

/* Solve every member from xs[k] (in: x0, out: x; n_k doubles each, host or
 * device per device_ptrs) with step length gammas[k] (NULL: all 1) to
 * tols[k] (NULL: run max_sweeps sweeps), measured as ||x-x*||/||x*|| when
 * x_trues[k] is given (x_trues or an entry may be NULL) else ||b-Ax||/||b||;
 * at most max_sweeps sweeps each.  infos (count entries, may be NULL) get
 * each problem's outcome; rel_res is the final FP64 ||b - A x||/||b||.  Each
 * problem's row sequence continues from its position, which advances.
 * Returns OK when all converged, else the worst status (NOT_CONVERGED,
 * DIVERGED), or EINVAL / ECUDA. */
int asyrk_batch_solve(asyrk_batch *b, double *const *xs, const double *gammas, const double *tols,
                      int64_t max_sweeps, const double *const *x_trues, int device_ptrs,
                      asyrk_solve_info *infos, asyrk_batch_info *binfo);

void asyrk_batch_destroy(asyrk_batch *b);

/* ------------------------------------------------------------------------
 * Served solves (not in the paper): continuous batching.  Requests name a
 * resident problem (FP32 or BF16 values) and bring x0, optionally x*, gamma,
 * a tolerance and a mode: ASYNC (FP32 iterate) or REFINE (FP64 iterate, each
 * outer step r = b - A x in FP64 then an FP32 inner solve of A d = r aimed at
 * a relative residual of inner_tol: checked at every engine step in the
 * shared step; on-chip, run for the sweep count that the previous outer
 * step's contraction says meets it, as asyrk_solve plans it).  An engine
 * thread admits queued requests into free slots while the device-memory
 * budget allows -- each request's iterate, staging, claim bits and residual,
 * plus its problem's bytes counted once while any request uses it -- and
 * advances the admitted requests together in engine steps of one kernel
 * launch, each step at least 512 projections per worker long, in which a
 * request runs as many whole sweeps as fit but no more than it is predicted
 * to still need; requests whose problem fits a CTA's shared memory are solved
 * on-chip instead, one CTA each, on SMs of their own (onchip, partition).  A
 * request that finishes frees its slot for the next.  Each request draws its
 * own row sequence (Philox stream = its ticket), so one problem can serve
 * several requests at once.  The problems must outlive their requests; the
 * server must outlive every wait on it.
 * ------------------------------------------------------------------------ */
typedef struct asyrk_server asyrk_server; /* opaque */

typedef struct asyrk_server_opts {
    int64_t mem_budget_bytes;  /* device bytes admitted requests may hold (> 0)      */
    int32_t max_slots;         /* requests in flight at once (0: 256)                */
    int32_t row_exclusion;     /* as in asyrk_solve_opts                             */
    double inner_tol;          /* REFINE inner target (0: 1e-3)                      */
    int64_t max_inner_sweeps;  /* REFINE inner sweeps per outer step at most (0: 60) */
    int32_t onchip;            /* >= 0: requests whose problem fits a CTA's shared
                                  memory are solved on-chip (default); -1: never     */
    int32_t partition;         /* with on-chip requests: the shared step and the
                                  on-chip requests on disjoint SMs, the on-chip ones
                                  on this many (0: 16; rounded up to the driver's
                                  granularity) where the driver offers SM partitions;
                                  -1: they share every SM (the step then takes three
                                  quarters of the resident warps while on-chip
                                  requests run)                                      */
    double admit_load;         /* shared-step admission: queued requests are admitted
                                  in arrival order while the warp demands of the
                                  requests in the step (each its Cor. 2 worker cap
                                  in warps, at most the resident warps) add up to at
                                  most admit_load x the resident warps; one request
                                  is always admitted.  0: 1.0; < 0: no limit (only
                                  slots and memory bound admission)                 */
} asyrk_server_opts;

typedef struct asyrk_server_stats {
    int64_t submitted, completed, queued, active;
    int64_t iterations;        /* engine steps run                                   */
    int64_t kernel_launches;   /* kernels the engine launched                        */
    int64_t mem_used;          /* bytes charged against the budget now               */
    int64_t mem_budget;
    int64_t arena_reserved;    /* bytes the arena holds from cudaMalloc              */
    int32_t max_slots;
    int32_t max_active;        /* most requests in flight at once so far             */
    int32_t fatal;             /* first hard error of the engine, or OK              */
    int32_t max_active_shared; /* most requests in the shared engine step at once    */
    int64_t onchip_completed;  /* requests solved on-chip so far                     */
    int32_t step_sms;          /* SMs of the shared step when split from the on-chip
                                  requests' SMs, else 0                              */
    int32_t onchip_sms;        /* SMs of the on-chip requests when split, else 0     */
} asyrk_server_stats;

/* Start a server on the current device.  Errors: EINVAL, ENOMEM, ECUDA. */
int asyrk_server_create(asyrk_server **out, const asyrk_server_opts *opts);

/* Queue a request; x0 (n doubles, NULL = zeros) and x_true (n doubles, NULL =
 * measure ||b - Ax||/||b||) are host arrays copied before the call returns.
 * The tolerance applies to ||x-x*||/||x*|| with x_true, else to the residual.
 * Errors: EINVAL (FP64 problem, mode not ASYNC/REFINE, gamma outside (0, 2),
 * tol <= 0, max_sweeps < 1, server stopping), ENOMEM (needs more than the whole
 * budget; nothing is queued). */
int asyrk_server_submit(asyrk_server *s, asyrk_problem *p, const double *x0,
                        const double *x_true, double gamma, double tol, int mode,
                        int64_t max_sweeps, uint64_t *ticket);

/* Wait up to timeout_us microseconds (< 0: no limit) for a request; on
 * completion copy its x (n doubles, may be NULL) and info (info.seconds = time
 * from submit to completion) and forget the ticket.  Returns the request's
 * status (OK, NOT_CONVERGED, DIVERGED, ECANCELED, or the engine's hard error),
 * ETIMEOUT (the ticket stays valid), or EINVAL (unknown ticket). */
int asyrk_server_wait(asyrk_server *s, uint64_t ticket, double *x, asyrk_solve_info *info,
                      int64_t timeout_us);

/* Cancel a request: a queued one completes at once, a running one at the
 * end of the current engine step, with status ECANCELED.  Errors: EINVAL. */
int asyrk_server_cancel(asyrk_server *s, uint64_t ticket);

int asyrk_server_get_stats(asyrk_server *s, asyrk_server_stats *stats);

/* Stop the engine; unfinished requests complete with ECANCELED and every
 * ticket is forgotten. */
void asyrk_server_destroy(asyrk_server *s);

/* ---- least squares (Section 6) ------------------------------------------
 * min ||A x - b|| for a possibly inconsistent A x = b is reached by the method
 * run on the square consistent system
 *     [ 0   phi A^T ] [x]   [phi A^T b]
 *     [ A   -zeta I ] [y] = [    0    ]
 * over z = (x, y) of length n + m, whose solutions have x = zeta x_LS and
 * y = A x_LS (from z0 = 0 the method reaches the minimum-norm one, so
 * x = zeta pinv(A) b).  Section 6 shows that phi = 1, zeta = sigma_r/sqrt(2)
 * (sigma_r the smallest nonzero singular value of A, rows of A normalised)
 * maximises lambda_min/||.||_F^2 of the system, the quantity the rate of
 * Theorem 2 depends on. */
typedef struct asyrk_lsq_opts {
    double zeta;           /* > 0: the y-block scale; 0: Section 6's sigma_r/sqrt(2)
                              with sigma_r from asyrk_spectrum_estimate            */
    double phi;            /* > 0: the A^T-block scale; 0 means 1                   */
    uint64_t seed;         /* Philox key of the system's row sequence (and of the
                              estimate's start vector)                              */
    int32_t device_ptrs;   /* 1: row_ptr, col_idx, values, b are device pointers    */
    int32_t lanczos_steps; /* steps of the sigma_r estimate when zeta = 0; 0: 100   */
    void *stream;          /* cudaStream_t for the set-up work; NULL = default      */
} asyrk_lsq_opts;

/* Create the problem of the system above from A (m x n CSR, as for
 * asyrk_create except that rows of A may be empty) and b (m doubles).  The
 * system has one row per non-empty column of A (entries (n + i, phi A_ij), i
 * ascending; right side phi sum_i A_ij b_i in FP64, ascending i, no fused
 * multiply-adds), then one per row i of A (a_i, then (n + i, -zeta); right
 * side 0); a column of zeros would give the row 0 = 0 and is left out.  Values
 * are stored in vdtype (phi A_ij and -zeta rounded to nearest; BF16 through
 * FP32); with FP32/BF16 values the A^T block is phi A exactly only when phi is
 * a power of two (phi = 1 is Section 6's choice), otherwise it carries the
 * rounding of phi A_ij.  Solve it with asyrk_solve on an iterate of n + m doubles, then read
 * x_LS with asyrk_lsq_solution.  Host arrays are read before the call returns.
 * Errors: EINVAL (m, n < 1, m + n > 2^31-1, more than 2^32-1 nonzeros, a
 * malformed CSR, non-finite data, zeta < 0, phi < 0, lanczos_steps < 0, opts
 * NULL, A without a nonzero when zeta = 0), ENOMEM, ECUDA.  On error *out is
 * NULL. */
int asyrk_lsq_create(asyrk_problem **out, int64_t m, int64_t n, const int64_t *row_ptr,
                     const int32_t *col_idx, const void *values, int vdtype, const double *b,
                     const asyrk_lsq_opts *opts);

/* x_LS = x-block of z / zeta_s for a problem made by asyrk_lsq_create, zeta_s
 * being zeta as the system stores it (rounded to vdtype, so that the identity
 * x = zeta_s x_LS is exact for the stored system); z has
 * n + m doubles, x_ls n doubles, both on the host or both on the device
 * (on_device).  Errors: EINVAL (NULL, not a least-squares problem), ENOMEM,
 * ECUDA. */
int asyrk_lsq_solution(asyrk_problem *p, const double *z, int on_device, double *x_ls);

/* zeta (as stored) and phi of a least-squares problem; either pointer may be
 * NULL.  Errors: EINVAL (NULL problem, not a least-squares problem). */
int asyrk_lsq_params(const asyrk_problem *p, double *zeta, double *phi);

/* Estimates of the smallest NONZERO eigenvalue and the largest eigenvalue of
 * A^T A (Section 1's lambda_min and lambda_max; sigma_r^2 of Section 6), from
 * `steps` Lanczos steps (0: 100) with full reorthogonalisation on the GPU,
 * started from A^T u with u a random sign vector (Philox, key seed), so the
 * Krylov space lies in the row space of A and null-space directions are left
 * out (Ritz values under 1e-10 lambda_max are passed over as rounding-level
 * null-space components).  Ritz values lie inside the spectrum: the estimates
 * satisfy lambda_min <= *lambda_min and *lambda_max <= lambda_max up to
 * rounding, and converge to them as steps grows (fast at both ends for the
 * random sparse matrices of Section 5 when m/n is away from 1).  A is an
 * m x n CSR as for asyrk_lsq_create (empty rows allowed), on the host or the
 * device (device_ptrs); work runs on `stream` (a cudaStream_t, NULL = default);
 * the device needs n (steps + 1) doubles for the Lanczos basis.
 * Errors: EINVAL (dimensions, malformed CSR, non-finite values, steps < 0,
 * A without a nonzero), ENOMEM, ECUDA. */
int asyrk_spectrum_estimate(int64_t m, int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                            const void *values, int vdtype, int device_ptrs, int32_t steps,
                            uint64_t seed, void *stream, double *lambda_min, double *lambda_max);

/* Largest m accepted by asyrk_residual_noalloc. */
#define ASYRK_NOALLOC_MAX_ROWS 16777216

/* ||b - A x||_2 (out[0]) and ||b||_2 (out[1]) in FP64 for a CSR system that the
 * caller holds in device memory, computed without allocating anything.  The
 * paper has no counterpart: this entry point is for callers that cannot call
 * cudaMalloc -- those whose device memory was all handed to their own pool or
 * arena up front (a service that must not hit out-of-memory mid-request) and
 * those on a latency-critical path where cudaMalloc/cudaFree would synchronise
 * the device.  asyrk_residual needs a problem handle, and creating one
 * allocates; this call needs only the caller's arrays.
 *   row_ptr (m+1 int64), col_idx (nnz int32), values (nnz of vdtype), b (m
 *   doubles), x (n doubles) and out (2 doubles) are all DEVICE pointers, in
 *   the plain CSR layout of asyrk_create.  Entries outside [0, nnz) and
 *   columns outside [0, n) are not read; they make out[0] NaN.
 *   The work is enqueued on `stream` (NULL: legacy default stream) and the
 *   call returns without waiting: out is valid once the stream gets there.
 * Scratch: a file-scope device array of 128 KiB + 64 B inside the library,
 * which every GPU that loads the library holds until the process exits.  No
 * cudaMalloc, cudaFree or allocating library routine is called.  The first
 * call on a device looks up that array's device address (a one-time set-up
 * per device); make that first call before any stream capture on the device.
 * All calls share the one array: calls whose GPU work overlaps (different
 * streams without ordering between them) race and give wrong results; order
 * them on one stream or wait in between.
 * Errors: EINVAL (m < 1 or m > ASYRK_NOALLOC_MAX_ROWS -- the rows the static
 * scratch can hold --, n outside [1, 2^31-1], nnz < 0, a NULL pointer, an
 * unknown vdtype), ECUDA. */
int asyrk_residual_noalloc(int64_t m, int64_t n, int64_t nnz, const int64_t *row_ptr,
                           const int32_t *col_idx, const void *values, int vdtype,
                           const double *b, const double *x, double *out, void *stream);

/* Static description of a status code. */
const char *asyrk_strerror(int status);

/* One-line description of the last hard error on the calling thread. */
const char *asyrk_last_error(void);

/* ASYRK_ABI_VERSION of the loaded library. */
int asyrk_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ASYRK_H */
