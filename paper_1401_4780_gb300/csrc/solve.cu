// solve.cu -- asyrk_solve and asyrk_residual: the host side of a solve.
//
// A solve alternates launches of the projection kernel (check_every sweeps of
// m projections each) with an FP64 check on the GPU, whose 8-byte result is
// the only thing read back per check.  The modes:
//   SEQUENTIAL  one worker, FP64 x, projections strictly in order (Eq. (2));
//   ASYNC       W lock-free workers (Section 3), x in FP64 for FP64 values
//               and FP32 otherwise;
//   REFINE      x64 in FP64; per outer step r = b - A x64 in FP64, the ASYNC
//               FP32 kernel solves A d = r for a number of inner sweeps, and
//               x64 += d.  The inner sweep count adapts so that each outer
//               step shrinks the residual by about inner_tol.
#include <math.h>
#include <string.h>

#include <chrono>

#include "batch.cuh"
#include "devmem.cuh"

namespace asyrk {

static double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

static long long tau_cap(const asyrk_problem *p) { return tau_cap_estimate(p->m, p->n); }

enum { MEAS_ERR = 0, MEAS_RES = 1, MEAS_NORMAL = 2 };

struct SolveCtx {
    asyrk_problem *p;
    cudaStream_t s;
    bool have_xt;
    int kind;       // MEAS_ERR: ||x-x*||/||x*||, MEAS_RES: ||b-Ax||/||b||, MEAS_NORMAL: ||A^T(Ax-b)||^2
    double ref;     // ||x*|| or ||b||
    bool profile;
    double project_ms = 0.0;
    int64_t launches = 0;
};

// one projection launch, optionally bracketed by events on the launch stream
static int project(SolveCtx &c, const ProjectLaunch &L)
{
    if (c.profile) ASYRK_CK(cudaEventRecord(c.p->ev[0], c.s));
    int st = ASYRK_OK;
    const unsigned long long m = (unsigned long long)c.p->m;
    if (L.sampling == ASYRK_SAMPLE_SHUFFLED && L.count > m - L.j0 % m) {
        // shuffled sweeps run one launch per sweep: within a sweep every row
        // comes once, so no worker finds its row held by a worker of the next
        // sweep (a skip would drop that row's visit for the sweep)
        ProjectLaunch one = L;
        unsigned long long done = 0;
        while (done < L.count && st == ASYRK_OK) {
            one.j0 = L.j0 + done;
            const unsigned long long to_boundary = m - one.j0 % m;
            one.count = L.count - done < to_boundary ? L.count - done : to_boundary;
            st = launch_project(one);
            done += one.count;
        }
    } else {
        st = launch_project(L);
    }
    if (st != ASYRK_OK) return st;
    if (c.profile) {
        ASYRK_CK(cudaEventRecord(c.p->ev[1], c.s));
        ASYRK_CK(cudaEventSynchronize(c.p->ev[1]));
        float ms = 0.f;
        ASYRK_CK(cudaEventElapsedTime(&ms, c.p->ev[0], c.p->ev[1]));
        c.project_ms += ms;
        c.launches += 1;
    }
    return ASYRK_OK;
}

// check measure of the iterate x (FP64 or FP32 on the device)
static int measure(SolveCtx &c, const void *x, bool x_f64, double *out)
{
    asyrk_problem *p = c.p;
    int st = c.kind == MEAS_ERR   ? launch_err2(p, x, x_f64, p->xt64, 0, c.s)
             : c.kind == MEAS_RES ? launch_residual(p, x, x_f64, false, 0, c.s)
                                  : launch_normal_residual(p, x, x_f64, 0, c.s);
    if (st != ASYRK_OK) return st;
    ASYRK_CK(cudaMemcpyAsync(p->h_out, p->red_out, 2 * sizeof(double), cudaMemcpyDeviceToHost, c.s));
    ASYRK_CK(cudaStreamSynchronize(c.s));
    *out = c.kind == MEAS_NORMAL ? p->h_out[0] : sqrt(p->h_out[0]) / c.ref;
    return ASYRK_OK;
}

static int final_residual(SolveCtx &c, const double *x64, double *rel_res)
{
    asyrk_problem *p = c.p;
    int st = launch_residual(p, x64, true, false, 0, c.s);
    if (st != ASYRK_OK) return st;
    ASYRK_CK(cudaMemcpyAsync(p->h_out, p->red_out, sizeof(double), cudaMemcpyDeviceToHost, c.s));
    ASYRK_CK(cudaStreamSynchronize(c.s));
    *rel_res = p->bnorm > 0.0 ? sqrt(p->h_out[0]) / p->bnorm : sqrt(p->h_out[0]);
    return ASYRK_OK;
}

// element-wise helpers that do not know the handle: count their kernels here
static int convert(asyrk_problem *p, const void *src, bool src_f64, void *dst, bool dst_f64,
                   cudaStream_t s)
{
    int st = launch_convert(src, src_f64, dst, dst_f64, p->n, s);
    if (st == ASYRK_OK && src_f64 != dst_f64) p->launches += 1;
    return st;
}

__host__ __device__ static bool diverged(double meas, double meas0)
{
    return !isfinite(meas) || meas > 1e30 * (meas0 > 0.0 ? meas0 : 1.0);
}

// Adaptive check interval (check_every = 0): from the contraction the last k
// sweeps achieved, rho = (meas / prev)^(1/k) per sweep, the sweeps still needed
// are log(tol / meas) / log(rho); the next check comes after half of them, at
// least 1 sweep, at most twice the last interval and at most a tenth of the
// sweeps done so far -- so a solve stops at most 10 % past the sweep where the
// tolerance was met, and checks O(log sweeps) times when the decay is steady.
// Without a measured contraction the interval is one sweep.
__host__ __device__ static int64_t next_check(double prev, double meas, int64_t k, int64_t done,
                                              double tol)
{
    int64_t cap = done / 10;
    if (cap < 1) cap = 1;
    if (cap > 2 * k) cap = 2 * k;
    if (!(tol > 0.0)) return cap;  // fixed sweep count: checks only watch for divergence
    if (!(meas > 0.0) || !(prev > meas) || !(meas > tol)) return 1;
    const double rho = pow(meas / prev, 1.0 / (double)k);
    if (!(rho > 0.0 && rho < 1.0)) return 1;
    const double need = log(tol / meas) / log(rho);
    double next = ceil(0.5 * need);
    if (next < 1.0) next = 1.0;
    if (next > (double)cap) next = (double)cap;
    return (int64_t)next;
}

// ---------------------------------------------------------------------------
// graph-captured solve loop: one CUDA-graph launch runs [k sweeps, the check,
// the decision] in a WHILE node until the decision kernel clears the
// condition, so the host waits once per solve instead of once per check
// ---------------------------------------------------------------------------
struct LoopState {
    unsigned long long j, count;  // read by the projection kernel (position, length)
    long long sweeps, k;          // sweeps done, sweeps in the coming launch
    double meas, meas0, meas_prev;
    int status, iters;
};
static_assert(sizeof(LoopState) == 8 * sizeof(double), "fits the pinned readback buffer");

__global__ void k_loop_decide(LoopState *st, const double *red_out, int kind, double ref,
                              double tol, long long m, long long max_sweeps, long long check_every,
                              cudaGraphConditionalHandle h)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double v = red_out[0];
    const double meas = kind == MEAS_NORMAL ? v : sqrt(v) / ref;
    st->j += st->count;
    st->sweeps += st->k;
    st->iters += 1;
    int status = ASYRK_NOT_CONVERGED;
    if (diverged(meas, st->meas0)) status = ASYRK_DIVERGED;
    else if (tol > 0.0 && meas <= tol) status = ASYRK_OK;
    long long next = check_every > 0 ? check_every
                                     : next_check(st->meas_prev, meas, st->k, st->sweeps, tol);
    const long long left = max_sweeps - st->sweeps;
    if (next > left) next = left;
    st->meas = meas;
    st->meas_prev = meas;
    st->status = status;
    st->k = next;
    st->count = (unsigned long long)next * (unsigned long long)m;
    cudaGraphSetConditional(h, (status == ASYRK_NOT_CONVERGED && left > 0) ? 1u : 0u);
}

static int loop_resources(asyrk_problem *p)
{
    if (!p->loop_state) {
        const int st = devmem_alloc(&p->loop_state, sizeof(LoopState), nullptr);
        if (st != ASYRK_OK) return st;
        ASYRK_CK(cudaStreamSynchronize(nullptr));  // in place before the loop's streams use it
        p->dev_bytes += (int64_t)sizeof(LoopState);
    }
    if (!p->cap_stream) ASYRK_CK(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
    return ASYRK_OK;
}

// Runs the loop from the state in *init (meas0 and the first k set) and
// returns the final state.  L describes the projection launch (its j0/count
// are replaced by the device words).
static int run_device_loop(SolveCtx &c, ProjectLaunch L, const LoopState &init, double tol,
                           int64_t max_sweeps, int64_t check_every, LoopState *out,
                           int64_t *launches_per_iter)
{
    asyrk_problem *p = c.p;
    int st = loop_resources(p);
    if (st != ASYRK_OK) return st;
    LoopState *dev = (LoopState *)p->loop_state;
    memcpy(p->h_out, &init, sizeof init);
    ASYRK_CK(cudaMemcpyAsync(dev, p->h_out, sizeof init, cudaMemcpyHostToDevice, c.s));
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    auto done = [&](int code) {
        if (exec) cudaGraphExecDestroy(exec);
        if (g) cudaGraphDestroy(g);
        return code;
    };
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return done(cuda_fail(e, "cudaGraphCreate", __FILE__, __LINE__));
    cudaGraphConditionalHandle handle;
    e = cudaGraphConditionalHandleCreate(&handle, g, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return done(cuda_fail(e, "cudaGraphConditionalHandleCreate", __FILE__, __LINE__));
    // cudaGraphNodeParams has no usable default constructor in C++: zeroed storage
    alignas(cudaGraphNodeParams) unsigned char storage[sizeof(cudaGraphNodeParams)];
    memset(storage, 0, sizeof storage);
    cudaGraphNodeParams &cp = *reinterpret_cast<cudaGraphNodeParams *>(storage);
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp);
    if (e != cudaSuccess) return done(cuda_fail(e, "cudaGraphAddNode", __FILE__, __LINE__));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(p->cap_stream, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return done(cuda_fail(e, "cudaStreamBeginCaptureToGraph", __FILE__, __LINE__));
    const int64_t l0 = p->launches;
    L.dyn = &dev->j;
    L.stream = p->cap_stream;
    st = launch_project(L);
    if (st == ASYRK_OK) {
        st = c.kind == MEAS_ERR   ? launch_err2(p, L.x, L.x_f64, p->xt64, 0, p->cap_stream)
             : c.kind == MEAS_RES ? launch_residual(p, L.x, L.x_f64, false, 0, p->cap_stream)
                                  : launch_normal_residual(p, L.x, L.x_f64, 0, p->cap_stream);
    }
    if (st == ASYRK_OK) {
        k_loop_decide<<<1, 1, 0, p->cap_stream>>>(dev, p->red_out, c.kind, c.ref, tol,
                                                  (long long)p->m, (long long)max_sweeps,
                                                  (long long)check_every, handle);
        p->launches += 1;
        if (cudaGetLastError() != cudaSuccess) st = set_error(ASYRK_ECUDA, "decision kernel launch");
    }
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(p->cap_stream, &captured);
    if (st != ASYRK_OK) return done(st);
    if (e != cudaSuccess) return done(cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__));
    *launches_per_iter = p->launches - l0;
    e = cudaGraphInstantiate(&exec, g, 0);
    if (e != cudaSuccess) return done(cuda_fail(e, "cudaGraphInstantiate", __FILE__, __LINE__));
    e = cudaGraphLaunch(exec, c.s);
    if (e != cudaSuccess) return done(cuda_fail(e, "cudaGraphLaunch", __FILE__, __LINE__));
    e = cudaMemcpyAsync(p->h_out, dev, sizeof(LoopState), cudaMemcpyDeviceToHost, c.s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.s);
    if (e != cudaSuccess) return done(cuda_fail(e, "graph loop", __FILE__, __LINE__));
    memcpy(out, p->h_out, sizeof *out);
    return done(ASYRK_OK);
}

static int solve_plain(SolveCtx &c, double gamma, double tol, int64_t max_sweeps,
                       const asyrk_solve_opts &o, asyrk_solve_info &info)
{
    asyrk_problem *p = c.p;
    const bool seq = o.mode == ASYRK_MODE_SEQUENTIAL;
    const bool x_f64 = seq || p->dtype == ASYRK_F64;
    int G = o.subwarp ? o.subwarp : choose_subwarp(p->max_len, p->nnz, p->m);
    double frac = 1.0;
    int tG = 0;
    if (!seq && o.subwarp == 0 && o.workers == 0 && tuned_shape(p->dtype, p->max_len, &tG, &frac))
        G = tG;  // the autotuner's shape for this kind of problem
    long long W = 1;
    if (!seq) {
        int maxw = 0;
        int st = project_max_workers(p, x_f64, G, &maxw);
        if (st != ASYRK_OK) return st;
        if (o.workers > 0) {
            W = o.workers;
        } else {
            W = (long long)(frac * maxw);
            if (W < 1) W = 1;
            const long long cap = tau_cap(p);
            if (W > cap) W = cap;
        }
    }
    info.workers = (int32_t)W;
    info.subwarp = G;
    if (!x_f64 && p->rec_b_is_residual) {
        int st = launch_restore_rec_b(p, c.s);
        if (st != ASYRK_OK) return st;
    }
    // the iterate: p->x64 holds x0 in FP64; work on p->xw in the kernel's precision
    int st = convert(p, p->x64, true, p->xw, x_f64, c.s);
    if (st != ASYRK_OK) return st;

    double meas0 = 0.0, meas = 0.0;
    if ((st = measure(c, p->xw, x_f64, &meas0)) != ASYRK_OK) return st;
    meas = meas0;
    int status = (tol > 0.0 && meas <= tol) ? ASYRK_OK : ASYRK_NOT_CONVERGED;
    int64_t sweeps = 0;
    const unsigned long long m = (unsigned long long)p->m;
    const bool adaptive = o.check_every == 0;
    int64_t k_next = 1;
    double meas_prev = meas0;
    // the device-driven loop when asked for, except with per-launch timing or
    // shuffled sweeps (which launch sweep by sweep)
    if (status == ASYRK_NOT_CONVERGED && max_sweeps > 0 && o.graph_loop && !c.profile &&
        o.sampling == ASYRK_SAMPLE_WEIGHTED) {
        ProjectLaunch L;
        L.p = p;
        L.x = p->xw;
        L.x_f64 = x_f64;
        L.gamma = gamma;
        L.stream_id = 0;
        L.workers = (int)W;
        L.subwarp = G;
        L.sequential = seq;
        L.exclusive = o.row_exclusion >= 0;
        L.sampling = o.sampling;
        L.update = o.update;
        L.form = o.kernel_form;
        L.b_from_rec = !x_f64;
        LoopState init;
        memset(&init, 0, sizeof init);
        init.k = adaptive ? 1 : (o.check_every < max_sweeps ? o.check_every : max_sweeps);
        init.j = p->j_next;
        init.count = (unsigned long long)init.k * m;
        init.meas = init.meas0 = init.meas_prev = meas0;
        init.status = ASYRK_NOT_CONVERGED;
        L.j0 = init.j;          // the kernel reads both from the loop state; a non-zero
        L.count = init.count;   // count keeps launch_project from skipping the launch
        LoopState fin;
        int64_t per_iter = 0;
        const int64_t l_before = p->launches;
        if ((st = run_device_loop(c, L, init, tol, max_sweeps, o.check_every, &fin, &per_iter)) !=
            ASYRK_OK)
            return st;
        p->launches = l_before + per_iter * fin.iters;
        p->j_next = fin.j;
        sweeps = fin.sweeps;
        info.projections += (int64_t)(fin.j - init.j);
        status = fin.status;
        meas = fin.meas;
    }
    while (status == ASYRK_NOT_CONVERGED && sweeps < max_sweeps) {
        int64_t k = adaptive ? k_next : o.check_every;
        if (k > max_sweeps - sweeps) k = max_sweeps - sweeps;
        ProjectLaunch L;
        L.p = p;
        L.x = p->xw;
        L.x_f64 = x_f64;
        L.gamma = gamma;
        L.j0 = p->j_next;
        L.count = (unsigned long long)k * m;
        L.stream_id = 0;
        L.workers = (int)W;
        L.subwarp = G;
        L.sequential = seq;
        L.exclusive = o.row_exclusion >= 0;
        L.sampling = o.sampling;
        L.update = o.update;
        L.form = o.kernel_form;
        L.b_from_rec = !x_f64;
        L.stream = c.s;
        if ((st = project(c, L)) != ASYRK_OK) return st;
        p->j_next += L.count;
        sweeps += k;
        info.projections += (int64_t)L.count;
        if ((st = measure(c, p->xw, x_f64, &meas)) != ASYRK_OK) return st;
        if (diverged(meas, meas0)) {
            status = ASYRK_DIVERGED;
            break;
        }
        if (tol > 0.0 && meas <= tol) status = ASYRK_OK;
        if (adaptive) k_next = next_check(meas_prev, meas, k, sweeps, tol);
        meas_prev = meas;
    }
    if (tol <= 0.0 && status == ASYRK_NOT_CONVERGED && sweeps == max_sweeps) status = ASYRK_OK;
    info.sweeps = sweeps;
    if ((st = convert(p, p->xw, x_f64, p->x64, true, c.s)) != ASYRK_OK) return st;
    return status;
}

static int solve_refine(SolveCtx &c, double gamma, double tol, int64_t max_sweeps,
                        const asyrk_solve_opts &o, asyrk_solve_info &info)
{
    asyrk_problem *p = c.p;
    int G = o.subwarp ? o.subwarp : choose_subwarp(p->max_len, p->nnz, p->m);
    double frac = 1.0;
    int tG = 0;
    if (o.subwarp == 0 && o.workers == 0 && tuned_shape(p->dtype, p->max_len, &tG, &frac)) G = tG;
    int maxw = 0;
    int st = project_max_workers(p, false, G, &maxw);
    if (st != ASYRK_OK) return st;
    long long W = o.workers > 0 ? o.workers : (long long)(frac * maxw);
    if (W < 1) W = 1;
    if (o.workers <= 0 && W > tau_cap(p)) W = tau_cap(p);
    info.workers = (int32_t)W;
    info.subwarp = G;
    const double inner_tol = o.inner_tol > 0.0 ? o.inner_tol : 1e-3;
    int64_t inner = o.inner_sweeps > 0 ? o.inner_sweeps : 8;
    float *d = (float *)p->xw;
    const unsigned long long m = (unsigned long long)p->m;

    double meas0 = -1.0, meas = 0.0, rprev = -1.0;
    int64_t sweeps = 0;
    int status = ASYRK_NOT_CONVERGED;
    for (;;) {
        // r = b - A x64 in FP64, stored as the inner right-hand side
        if ((st = launch_residual(p, p->x64, true, true, 0, c.s)) != ASYRK_OK) return st;
        if (c.kind == MEAS_ERR && (st = launch_err2(p, p->x64, true, p->xt64, 2, c.s)) != ASYRK_OK)
            return st;
        if (c.kind == MEAS_NORMAL && (st = launch_normal_residual(p, p->x64, true, 2, c.s)) != ASYRK_OK)
            return st;
        ASYRK_CK(cudaMemcpyAsync(p->h_out, p->red_out, 4 * sizeof(double), cudaMemcpyDeviceToHost, c.s));
        ASYRK_CK(cudaStreamSynchronize(c.s));
        const double rnorm = sqrt(p->h_out[0]);
        meas = c.kind == MEAS_ERR   ? sqrt(p->h_out[2]) / c.ref
               : c.kind == MEAS_RES ? rnorm / c.ref
                                    : p->h_out[2];
        if (meas0 < 0.0) meas0 = meas;
        if (diverged(meas, meas0)) { status = ASYRK_DIVERGED; break; }
        if (tol > 0.0 && meas <= tol) { status = ASYRK_OK; break; }
        if (sweeps >= max_sweeps) break;
        // this step's inner target: inner_tol, or, when the tolerance is
        // closer than that, just the reduction it still needs (with a margin
        // of 2), so the last inner solve does not overshoot the tolerance
        double step_tol = inner_tol;
        if (tol > 0.0 && (c.kind == MEAS_ERR || c.kind == MEAS_RES) && meas > 0.0) {
            const double need = 0.5 * tol / meas;
            if (need > step_tol) step_tol = need < 0.5 ? need : 0.5;
        }
        if (o.inner_sweeps <= 0 && rprev > 0.0 && rnorm > 0.0) {
            // adapt the inner sweep count to the contraction the last step achieved
            const double rho = rnorm / rprev;
            if (rho > 0.0 && rho < 1.0) {
                double want = (double)inner * log(step_tol) / log(rho);
                if (want < 2.0) want = 2.0;
                if (want > 4.0 * inner) want = 4.0 * inner;
                inner = (int64_t)ceil(want);
            } else {
                inner *= 2;
            }
            if (inner > 1000) inner = 1000;
        }
        rprev = rnorm;
        if (rnorm == 0.0) { status = ASYRK_OK; break; }
        int64_t k = inner;
        if (k > max_sweeps - sweeps) k = max_sweeps - sweeps;
        ASYRK_CK(cudaMemsetAsync(d, 0, p->n * sizeof(float), c.s));
        ProjectLaunch L;
        L.p = p;
        L.x = d;
        L.x_f64 = false;
        L.gamma = gamma;
        L.j0 = p->j_next;
        L.count = (unsigned long long)k * m;
        L.stream_id = 0;
        L.workers = (int)W;
        L.subwarp = G;
        L.sequential = false;
        L.exclusive = o.row_exclusion >= 0;
        L.sampling = o.sampling;
        L.update = o.update;
        L.form = o.kernel_form;
        L.b_from_rec = true;
        L.stream = c.s;
        if ((st = project(c, L)) != ASYRK_OK) return st;
        p->j_next += L.count;
        sweeps += k;
        info.projections += (int64_t)L.count;
        if ((st = launch_axpy_f32_to_f64(p->x64, d, p->n, c.s)) != ASYRK_OK) return st;
        p->launches += 1;
        info.refine_steps += 1;
    }
    if (tol <= 0.0 && status == ASYRK_NOT_CONVERGED && sweeps >= max_sweeps) status = ASYRK_OK;
    info.sweeps = sweeps;
    if ((st = launch_restore_rec_b(p, c.s)) != ASYRK_OK) return st;
    return status;
}

}  // namespace asyrk

using namespace asyrk;

extern "C" int asyrk_solve(asyrk_problem *p, double *x, double gamma, double tol,
                           int64_t max_sweeps, const asyrk_solve_opts *opts,
                           asyrk_solve_info *info_out)
{
    const double t0 = now_s();
    asyrk_solve_info info;
    memset(&info, 0, sizeof info);
    info.rel_err = -1.0;
    if (info_out) *info_out = info;
    if (!p || !x) return set_error(ASYRK_EINVAL, "NULL problem or x");
    if (!(gamma > 0.0 && gamma < 2.0)) return set_error(ASYRK_EINVAL, "gamma must be in (0, 2)");
    if (max_sweeps < 0) return set_error(ASYRK_EINVAL, "max_sweeps < 0");
    asyrk_solve_opts o;
    memset(&o, 0, sizeof o);
    o.mode = ASYRK_MODE_ASYNC;
    o.check_every = 1;
    if (opts) o = *opts;
    if (o.mode < ASYRK_MODE_SEQUENTIAL || o.mode > ASYRK_MODE_REFINE)
        return set_error(ASYRK_EINVAL, "unknown mode %d", o.mode);
    if (o.check_every < 0) return set_error(ASYRK_EINVAL, "check_every must be >= 0");
    if (o.workers < 0) return set_error(ASYRK_EINVAL, "workers < 0");
    if (o.subwarp != 0 && o.subwarp != 1 && o.subwarp != 2 && o.subwarp != 4 && o.subwarp != 8 &&
        o.subwarp != 16 && o.subwarp != 32)
        return set_error(ASYRK_EINVAL, "subwarp must be 0, 1, 2, 4, 8, 16 or 32");
    if (o.row_exclusion < -1 || o.row_exclusion > 1)
        return set_error(ASYRK_EINVAL, "row_exclusion must be -1, 0 or 1");
    if (o.measure < ASYRK_MEASURE_AUTO || o.measure > ASYRK_MEASURE_NORMAL_RESIDUAL)
        return set_error(ASYRK_EINVAL, "unknown measure %d", o.measure);
    if (o.sampling < ASYRK_SAMPLE_WEIGHTED || o.sampling > ASYRK_SAMPLE_SHUFFLED)
        return set_error(ASYRK_EINVAL, "unknown sampling %d", o.sampling);
    if (o.update < ASYRK_UPDATE_ROW || o.update > ASYRK_UPDATE_SINGLE)
        return set_error(ASYRK_EINVAL, "unknown update %d", o.update);
    if (o.graph_loop < 0 || o.graph_loop > 1) return set_error(ASYRK_EINVAL, "graph_loop must be 0 or 1");
    if (o.kernel_form < -1 || o.kernel_form > 1)
        return set_error(ASYRK_EINVAL, "kernel_form must be -1, 0 or 1");
    if (o.kernel_form == 1 && o.update == ASYRK_UPDATE_SINGLE)
        return set_error(ASYRK_EINVAL, "the latency form applies full-row updates only");
    if (o.mode == ASYRK_MODE_SEQUENTIAL && o.workers > 1)
        return set_error(ASYRK_EINVAL, "SEQUENTIAL mode has one worker");

    int st = ensure_workspace(p);
    if (st != ASYRK_OK) return st;
    const int64_t launches0 = p->launches;
    SolveCtx c;
    c.p = p;
    c.s = (cudaStream_t)o.stream;
    ASYRK_CK(cudaMemsetAsync(p->skipped, 0, sizeof(unsigned long long), c.s));
    c.profile = o.profile != 0;
    const cudaMemcpyKind in_kind = o.device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    ASYRK_CK(cudaMemcpyAsync(p->x64, x, p->n * sizeof(double), in_kind, c.s));
    c.have_xt = o.x_true != nullptr;
    c.kind = o.measure == ASYRK_MEASURE_NORMAL_RESIDUAL ? MEAS_NORMAL
             : (o.measure == ASYRK_MEASURE_RESIDUAL || !c.have_xt) ? MEAS_RES
                                                                   : MEAS_ERR;
    if (c.have_xt) {
        ASYRK_CK(cudaMemcpyAsync(p->xt64, o.x_true, p->n * sizeof(double), in_kind, c.s));
        if ((st = launch_sumsq(p, p->xt64, p->n, 4, c.s)) != ASYRK_OK) return st;
        ASYRK_CK(cudaMemcpyAsync(p->h_out + 4, p->red_out + 4, sizeof(double), cudaMemcpyDeviceToHost, c.s));
        ASYRK_CK(cudaStreamSynchronize(c.s));
        c.ref = sqrt(p->h_out[4]);
    }
    if (c.kind != MEAS_ERR) c.ref = p->bnorm;
    if (!(c.ref > 0.0)) c.ref = 1.0;

    int status = (o.mode == ASYRK_MODE_REFINE) ? solve_refine(c, gamma, tol, max_sweeps, o, info)
                                               : solve_plain(c, gamma, tol, max_sweeps, o, info);
    if (status < 0) {
        if (info_out) { info.status = status; *info_out = info; }
        return status;
    }
    // x64 now holds the final iterate in FP64
    if (c.have_xt) {
        if ((st = launch_err2(p, p->x64, true, p->xt64, 0, c.s)) != ASYRK_OK) return st;
        ASYRK_CK(cudaMemcpyAsync(p->h_out, p->red_out, sizeof(double), cudaMemcpyDeviceToHost, c.s));
        ASYRK_CK(cudaStreamSynchronize(c.s));
        info.rel_err = sqrt(p->h_out[0]) / c.ref;
    }
    if ((st = final_residual(c, p->x64, &info.rel_res)) != ASYRK_OK) return st;
    ASYRK_CK(cudaMemcpyAsync(p->h_out + 6, p->skipped, sizeof(unsigned long long),
                             cudaMemcpyDeviceToHost, c.s));
    const cudaMemcpyKind out_kind = o.device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    ASYRK_CK(cudaMemcpyAsync(x, p->x64, p->n * sizeof(double), out_kind, c.s));
    ASYRK_CK(cudaStreamSynchronize(c.s));
    {
        unsigned long long sk;
        memcpy(&sk, p->h_out + 6, sizeof sk);
        info.skipped = (int64_t)sk;
    }
    info.status = status;
    info.project_ms = c.project_ms;
    info.project_launches = c.launches;
    info.j_end = p->j_next;
    info.kernel_launches = p->launches - launches0;
    info.seconds = now_s() - t0;
    if (info_out) *info_out = info;
    return status;
}

extern "C" int asyrk_residual(asyrk_problem *p, const double *x, int x_on_device,
                              double *rel_residual)
{
    if (!p || !x || !rel_residual) return set_error(ASYRK_EINVAL, "NULL argument");
    int st = ensure_workspace(p);
    if (st != ASYRK_OK) return st;
    ASYRK_CK(cudaMemcpy(p->x64, x, p->n * sizeof(double),
                        x_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice));
    SolveCtx c;
    c.p = p;
    c.s = 0;
    c.have_xt = false;
    c.kind = MEAS_RES;
    c.ref = 1.0;
    c.profile = false;
    return final_residual(c, p->x64, rel_residual);
}

extern "C" int asyrk_normal_residual(asyrk_problem *p, const double *x, int x_on_device,
                                     double *value)
{
    if (!p || !x || !value) return set_error(ASYRK_EINVAL, "NULL argument");
    int st = ensure_workspace(p);
    if (st != ASYRK_OK) return st;
    ASYRK_CK(cudaMemcpy(p->x64, x, p->n * sizeof(double),
                        x_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice));
    if ((st = launch_normal_residual(p, p->x64, true, 0, 0)) != ASYRK_OK) return st;
    ASYRK_CK(cudaMemcpy(p->h_out, p->red_out, sizeof(double), cudaMemcpyDeviceToHost));
    *value = p->h_out[0];
    return ASYRK_OK;
}
