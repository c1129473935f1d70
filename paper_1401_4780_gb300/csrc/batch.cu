// batch.cu -- asyrk_batch_*: many independent systems solved by one graph launch.
//
// asyrk_batch_create fixes the member problems, picks each one's sub-warp
// width (the autotuner's choice for its row length when tuned, else one
// 4-entry chunk per lane) and its worker cap (the Cor. 2 estimate), lays out
// the per-slot buffers and captures the whole solve as a CUDA graph whose only
// top-level node is a WHILE conditional over one engine iteration (plan,
// project, check, cond; see batch.cuh).  The loop stops on the device when no
// slot is active or after the iteration bound, so asyrk_batch_solve is: copy
// inputs, one measure launch, one graph launch, copy results.
#include <math.h>
#include <string.h>

#include <chrono>
#include <set>
#include <vector>

#include "batch.cuh"

struct asyrk_batch {
    int count = 0;
    int device = 0;
    int resident_warps = 0;
    bool excl = true;
    bool graph = true;
    cudaStream_t user_stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    std::vector<asyrk_problem *> probs;
    std::vector<asyrk::SysDesc> h;       // host mirror of the table
    std::vector<int64_t> xoff;           // slot offsets into the x buffers
    int64_t n_total = 0;
    int total_chunks = 0;
    asyrk::SysDesc *d = nullptr;
    float *x = nullptr;
    double *x64 = nullptr;
    double *xt = nullptr;
    unsigned *busy = nullptr;
    double *part = nullptr;
    int *d_active = nullptr;
    int *d_iter = nullptr;
    int *h_ints = nullptr;  // pinned: active, iter
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    int64_t launches_per_iter = 4;
};

using namespace asyrk;

static void batch_free(asyrk_batch *b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->g) cudaGraphDestroy(b->g);
    cudaFree(b->d);
    cudaFree(b->x);
    cudaFree(b->x64);
    cudaFree(b->xt);
    cudaFree(b->busy);
    cudaFree(b->part);
    cudaFree(b->d_active);
    cudaFree(b->d_iter);
    if (b->h_ints) cudaFreeHost(b->h_ints);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->ev[0]) cudaEventDestroy(b->ev[0]);
    if (b->ev[1]) cudaEventDestroy(b->ev[1]);
    delete b;
}

static int build_graph(asyrk_batch *b)
{
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (b->g) {
        cudaGraphDestroy(b->g);
        b->g = nullptr;
    }
    ASYRK_CK(cudaGraphCreate(&b->g, 0));
    cudaGraphConditionalHandle handle;
    ASYRK_CK(cudaGraphConditionalHandleCreate(&handle, b->g, 1, cudaGraphCondAssignDefault));
    // cudaGraphNodeParams has no usable default constructor in C++: zeroed storage
    alignas(cudaGraphNodeParams) unsigned char storage[sizeof(cudaGraphNodeParams)];
    memset(storage, 0, sizeof storage);
    cudaGraphNodeParams &cp = *reinterpret_cast<cudaGraphNodeParams *>(storage);
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    ASYRK_CK(cudaGraphAddNode(&node, b->g, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    ASYRK_CK(cudaStreamBeginCaptureToGraph(b->cap_stream, body, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeRelaxed));
    int st = launch_batch_iteration(b->d, b->count, b->total_chunks, b->part, b->resident_warps,
                                    b->excl, b->d_active, b->d_iter, true,
                                    (unsigned long long)handle, b->cap_stream);
    cudaGraph_t captured = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->cap_stream, &captured);
    if (st != ASYRK_OK) return st;
    ASYRK_CK(e);
    ASYRK_CK(cudaGraphInstantiate(&b->exec, b->g, 0));
    return ASYRK_OK;
}

extern "C" int asyrk_batch_create(asyrk_batch **out, asyrk_problem *const *problems, int count,
                                  const asyrk_batch_opts *opts)
{
    if (!out) return set_error(ASYRK_EINVAL, "out is NULL");
    *out = nullptr;
    if (count < 1 || !problems) return set_error(ASYRK_EINVAL, "need at least one problem");
    asyrk_batch_opts o;
    memset(&o, 0, sizeof o);
    if (opts) o = *opts;
    if (o.row_exclusion < -1 || o.row_exclusion > 1)
        return set_error(ASYRK_EINVAL, "row_exclusion must be -1, 0 or 1");
    if (o.sampling < ASYRK_SAMPLE_WEIGHTED || o.sampling > ASYRK_SAMPLE_SHUFFLED ||
        o.update < ASYRK_UPDATE_ROW || o.update > ASYRK_UPDATE_SINGLE)
        return set_error(ASYRK_EINVAL, "unknown sampling or update");
    std::set<asyrk_problem *> seen;
    int dev = -1;
    ASYRK_CK(cudaGetDevice(&dev));
    for (int k = 0; k < count; ++k) {
        asyrk_problem *p = problems[k];
        if (!p) return set_error(ASYRK_EINVAL, "problem %d is NULL", k);
        if (p->dtype == ASYRK_F64)
            return set_error(ASYRK_EINVAL, "batched solves take FP32 or BF16 values (problem %d is FP64)", k);
        if (p->device != dev) return set_error(ASYRK_EINVAL, "problem %d lives on another device", k);
        if (!seen.insert(p).second) return set_error(ASYRK_EINVAL, "problem %d appears twice", k);
    }
    asyrk_batch *b = new (std::nothrow) asyrk_batch();
    if (!b) return set_error(ASYRK_ENOMEM, "host allocation failed");
    b->count = count;
    b->device = dev;
    b->excl = o.row_exclusion >= 0;
    b->graph = o.graph >= 0;
    b->user_stream = (cudaStream_t)o.stream;
    b->probs.assign(problems, problems + count);
    auto fail = [&](int st) {
        batch_free(b);
        return st;
    };
    int sms = problems[0]->sm_count;
    int st = batch_resident_warps(sms, b->excl, &b->resident_warps);
    if (st != ASYRK_OK) return fail(st);
    if (count > b->resident_warps || count > BATCH_MAX_SLOTS)
        return fail(set_error(ASYRK_EINVAL, "%d problems exceed the %d a batch can hold", count,
                              b->resident_warps < BATCH_MAX_SLOTS ? b->resident_warps
                                                                 : BATCH_MAX_SLOTS));

    b->h.assign(count, SysDesc());
    b->xoff.assign(count + 1, 0);
    int64_t busy_total = 0;
    std::vector<int64_t> busy_off(count);
    int chunks = 0;
    for (int k = 0; k < count; ++k) {
        asyrk_problem *p = problems[k];
        SysDesc &D = b->h[k];
        memset(&D, 0, sizeof D);
        const int G = engine_subwarp(p, true);
        const long long capw = tau_cap_estimate(p->m, p->n);
        D.G = G;
        long long cw = (capw * G + 31) / 32;
        D.cap_warps = (int)(cw < 1 ? 1 : cw > 0x7fffffff ? 0x7fffffff : cw);
        D.m = (unsigned)p->m;
        D.n = (unsigned)p->n;
        D.dtype = p->dtype;
        D.uniform = p->uniform;
        D.work = (double)p->nnz;
        D.key = make_uint2((unsigned)p->seed, (unsigned)(p->seed >> 32));
        D.rec = p->rec;
        D.col = p->col;
        D.val = p->val;
        D.b64 = p->b64;
        D.sampling = o.sampling;
        D.update = o.update;
        D.shuf_h = shuffle_half_bits(p->m);
        b->xoff[k + 1] = b->xoff[k] + p->n;
        busy_off[k] = busy_total;
        busy_total += (p->m + 31) / 32;
        const int64_t ce = (p->n + BATCH_ERR_CHUNK - 1) / BATCH_ERR_CHUNK;
        const int64_t cr = (p->m + BATCH_ROW_CHUNK - 1) / BATCH_ROW_CHUNK;
        D.chunk0 = chunks;
        D.nchunks = (int)(ce > cr ? ce : cr);
        chunks += D.nchunks;
    }
    b->n_total = b->xoff[count];
    b->total_chunks = chunks;
    cudaError_t e = cudaMalloc((void **)&b->d, count * sizeof(SysDesc));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->x, b->n_total * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->x64, b->n_total * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->xt, b->n_total * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->busy, busy_total * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->part, 2 * (size_t)chunks * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_active, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_iter, 2 * sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&b->h_ints, 4 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(b->busy, 0, busy_total * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev[1]);
    if (e != cudaSuccess) return fail(cuda_fail(e, "batch allocation", __FILE__, __LINE__));
    for (int k = 0; k < count; ++k) {
        b->h[k].x = b->x + b->xoff[k];
        b->h[k].x64 = b->x64 + b->xoff[k];
        b->h[k].busy = b->busy + busy_off[k];
    }
    if (b->graph && (st = build_graph(b)) != ASYRK_OK) return fail(st);
    *out = b;
    return ASYRK_OK;
}

extern "C" void asyrk_batch_destroy(asyrk_batch *b) { batch_free(b); }

extern "C" int asyrk_batch_solve(asyrk_batch *b, double *const *xs, const double *gammas,
                                 const double *tols, int64_t max_sweeps,
                                 const double *const *x_trues, int device_ptrs,
                                 asyrk_solve_info *infos, asyrk_batch_info *binfo)
{
    const auto t_start = std::chrono::steady_clock::now();
    if (!b || !xs) return set_error(ASYRK_EINVAL, "NULL batch or xs");
    if (max_sweeps < 0) return set_error(ASYRK_EINVAL, "max_sweeps < 0");
    if (binfo) memset(binfo, 0, sizeof *binfo);
    cudaStream_t s = b->user_stream;
    const cudaMemcpyKind in_kind = device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    for (int k = 0; k < b->count; ++k) {
        const double g = gammas ? gammas[k] : 1.0;
        if (!(g > 0.0 && g < 2.0)) return set_error(ASYRK_EINVAL, "gamma of problem %d outside (0, 2)", k);
        if (!xs[k]) return set_error(ASYRK_EINVAL, "x of problem %d is NULL", k);
        SysDesc &D = b->h[k];
        asyrk_problem *p = b->probs[k];
        D.gamma = (float)g;
        D.tol = tols ? tols[k] : 0.0;
        D.max_sweeps = max_sweeps;
        D.j = p->j_next;
        D.stream_id = 0;
        D.bvec = nullptr;
        D.skipped = 0;
        D.sweeps = 0;
        D.active = 1;
        D.status = ASYRK_NOT_CONVERGED;
        D.meas = D.meas0 = -1.0;
        D.first_nwarps = 0;
        D.nwarps = 0;
        D.max_k = 1;  // every sweep is checked: sweep counts comparable with a single solve
        D.k = 1;
        D.warp0 = 0;
        D.chk_count = 0;
        D.res_count = 0;
        const bool has_xt = x_trues && x_trues[k];
        D.xt = has_xt ? b->xt + b->xoff[k] : nullptr;
        D.ref = has_xt ? -1.0 : (p->bnorm > 0.0 ? p->bnorm : 1.0);
        ASYRK_CK(cudaMemcpyAsync(b->x64 + b->xoff[k], xs[k], p->n * sizeof(double), in_kind, s));
        if (has_xt)
            ASYRK_CK(cudaMemcpyAsync(b->xt + b->xoff[k], x_trues[k], p->n * sizeof(double),
                                     in_kind, s));
        if (p->rec_b_is_residual) {
            int st = launch_restore_rec_b(p, s);
            if (st != ASYRK_OK) return st;
        }
    }
    int st = launch_batch_convert(b->x64, b->x, b->n_total, true, s);
    if (st != ASYRK_OK) return st;
    ASYRK_CK(cudaMemcpyAsync(b->d, b->h.data(), b->count * sizeof(SysDesc), cudaMemcpyHostToDevice, s));
    const int max_iter = (int)(max_sweeps < 0x3ffffffe ? max_sweeps + 1 : 0x3fffffff);
    b->h_ints[2] = 0;
    b->h_ints[3] = max_iter;
    ASYRK_CK(cudaMemcpyAsync(b->d_iter, b->h_ints + 2, 2 * sizeof(int), cudaMemcpyHostToDevice, s));
    if ((st = launch_batch_measure(b->d, b->count, b->total_chunks, b->part, s)) != ASYRK_OK) return st;
    int64_t launches = 3;  // convert, measure, and the final convert below
    int64_t iters = 0;
    ASYRK_CK(cudaEventRecord(b->ev[0], s));
    if (b->graph) {
        ASYRK_CK(cudaGraphLaunch(b->exec, s));
        ASYRK_CK(cudaMemcpyAsync(b->h_ints + 1, b->d_iter, sizeof(int), cudaMemcpyDeviceToHost, s));
        ASYRK_CK(cudaStreamSynchronize(s));
        iters = b->h_ints[1];
    } else {
        for (int it = 0; it < max_iter; ++it) {
            if ((st = launch_batch_iteration(b->d, b->count, b->total_chunks, b->part,
                                             b->resident_warps, b->excl, b->d_active, b->d_iter,
                                             false, 0ull, s)) != ASYRK_OK)
                return st;
            ASYRK_CK(cudaMemcpyAsync(b->h_ints, b->d_active, sizeof(int), cudaMemcpyDeviceToHost, s));
            ASYRK_CK(cudaStreamSynchronize(s));
            ++iters;
            if (b->h_ints[0] == 0) break;
        }
    }
    ASYRK_CK(cudaEventRecord(b->ev[1], s));
    launches += 4 * iters;
    // results: x back to FP64, the final FP64 residual, the table
    if ((st = launch_batch_convert(b->x64, b->x, b->n_total, false, s)) != ASYRK_OK) return st;
    if ((st = launch_batch_residual(b->d, b->count, b->total_chunks, b->part, s)) != ASYRK_OK) return st;
    launches += 1;
    ASYRK_CK(cudaMemcpyAsync(b->h.data(), b->d, b->count * sizeof(SysDesc), cudaMemcpyDeviceToHost, s));
    const cudaMemcpyKind out_kind = device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    for (int k = 0; k < b->count; ++k)
        ASYRK_CK(cudaMemcpyAsync(xs[k], b->x64 + b->xoff[k], b->probs[k]->n * sizeof(double),
                                 out_kind, s));
    ASYRK_CK(cudaStreamSynchronize(s));
    float ms = 0.f;
    ASYRK_CK(cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]));
    const double secs =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    int worst = ASYRK_OK, converged = 0;
    int64_t projections = 0;
    for (int k = 0; k < b->count; ++k) {
        const SysDesc &D = b->h[k];
        asyrk_problem *p = b->probs[k];
        p->j_next = D.j;
        const int64_t proj = D.sweeps * (int64_t)D.m;
        projections += proj;
        if (D.status == ASYRK_OK) ++converged;
        if (D.status != ASYRK_OK && (worst == ASYRK_OK || D.status > worst)) worst = D.status;
        if (infos) {
            asyrk_solve_info &I = infos[k];
            memset(&I, 0, sizeof I);
            I.status = D.status;
            I.workers = D.first_nwarps * (32 / D.G);
            I.subwarp = D.G;
            I.sweeps = D.sweeps;
            I.projections = proj;
            I.seconds = secs;
            I.rel_err = D.xt ? D.meas : -1.0;
            I.rel_res = D.bb2 > 0.0 ? sqrt(D.res2 / D.bb2) : sqrt(D.res2);
            I.j_end = D.j;
            I.skipped = (int64_t)D.skipped;
        }
    }
    if (binfo) {
        binfo->status = worst;
        binfo->converged = converged;
        binfo->iterations = iters;
        binfo->projections = projections;
        binfo->seconds = secs;
        binfo->device_ms = ms;
        binfo->kernel_launches = launches;
        binfo->resident_warps = b->resident_warps;
        binfo->graph = b->graph ? 1 : 0;
    }
    return worst;
}
