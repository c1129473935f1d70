// batch.cu -- asyrk_batch_*: many independent systems solved by graph launches.
//
// asyrk_batch_create fixes the member problems, picks each one's sub-warp
// width (the autotuner's choice for its row length when tuned, else one
// 4-entry chunk per lane) and its worker cap (the Cor. 2 estimate), and splits
// the members between two engines:
//   * on-chip (cluster.cu): a member whose iterate fits a CTA's shared memory
//     is solved start to finish by one CTA; these launches are the nodes of
//     one CUDA graph;
//   * global iterate (batch.cuh, engine.cu): the other members, advanced
//     together by the multi-system engine; its whole loop is one CUDA graph
//     whose only top-level node is a WHILE conditional over one engine
//     iteration (plan, project, check, cond), stopped on the device when no
//     slot is active or after the iteration bound.
// The largest members that fit still go to the global engine while that
// shortens the estimated batch time (plan_members).  When both engines run,
// the SMs are split between them (partition.cuh): the on-chip engine gets
// enough SMs for its members' thread-time within 1/2.5 of its longest member's
// solve, the global engine the rest, each on its own stream.  asyrk_batch_solve:
// copy inputs, launch both graphs at once, copy results.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <numeric>
#include <set>
#include <vector>

#include "batch.cuh"
#include "cluster.cuh"
#include "partition.cuh"

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
    // the on-chip engine: members whose iterate fits a CTA's shared memory
    std::vector<char> on;                // per member: 1 on-chip, 0 global-iterate engine
    int n_on = 0, n_glob = 0;
    std::vector<asyrk::ClusterShape> shapes;
    std::vector<asyrk::ClusterJob> hj;   // host mirror of the job table
    asyrk::ClusterJob *jobs = nullptr;
    std::vector<int> order;              // on-chip members, longest estimated solve first
    cudaGraph_t g_on = nullptr;
    cudaGraphExec_t exec_on = nullptr;
    cudaStream_t side = nullptr;         // the global engine's stream when both run
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // both engines at once: the SMs split between them (stream 0 global, 1 on-chip)
    asyrk::SmPartition split;
    int resident_warps_glob = 0;         // the global engine's warps on its SMs
    int *onchip_list = nullptr;          // device: on-chip members grouped per launch
    cudaEvent_t ev_on_join = nullptr;
    cudaEvent_t ev_done[2] = {nullptr, nullptr};  // end of the global / on-chip part (timed)
};

using namespace asyrk;

static void batch_free(asyrk_batch *b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->g) cudaGraphDestroy(b->g);
    if (b->exec_on) cudaGraphExecDestroy(b->exec_on);
    if (b->g_on) cudaGraphDestroy(b->g_on);
    if (b->side) cudaStreamDestroy(b->side);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_join) cudaEventDestroy(b->ev_join);
    if (b->ev_on_join) cudaEventDestroy(b->ev_on_join);
    for (cudaEvent_t e : b->ev_done)
        if (e) cudaEventDestroy(e);
    sm_partition_destroy(&b->split);
    cudaFree(b->onchip_list);
    cudaFree(b->d);
    cudaFree(b->x);
    cudaFree(b->x64);
    cudaFree(b->xt);
    cudaFree(b->busy);
    cudaFree(b->part);
    cudaFree(b->d_active);
    cudaFree(b->d_iter);
    cudaFree(b->jobs);
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
    const int warps = b->resident_warps_glob > 0 ? b->resident_warps_glob : b->resident_warps;
    int st = launch_batch_iteration(b->d, b->count, b->total_chunks, b->part, warps,
                                    b->excl, b->d_active, b->d_iter, true,
                                    (unsigned long long)handle, b->cap_stream);
    cudaGraph_t captured = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->cap_stream, &captured);
    if (st != ASYRK_OK) return st;
    ASYRK_CK(e);
    ASYRK_CK(cudaGraphInstantiate(&b->exec, b->g, 0));
    return ASYRK_OK;
}

// The on-chip engine's graph: one kernel node per on-chip member, no
// dependencies, the longest estimated solves placed first.
static int build_onchip_graph(asyrk_batch *b, bool grouped)
{
    ASYRK_CK(cudaGraphCreate(&b->g_on, 0));
    if (!grouped) {
        for (int k : b->order) {
            int st = cluster_add_node(b->g_on, b->probs[k]->dtype, b->shapes[k], b->jobs, k);
            if (st != ASYRK_OK) return st;
        }
        ASYRK_CK(cudaGraphInstantiate(&b->exec_on, b->g_on, 0));
        return ASYRK_OK;
    }
    // members with the same value type and sub-warp width, and threads and
    // shared memory in the same bucket (threads to a multiple of 128, memory to
    // a power of two from 8 KiB), share one launch whose CTA b solves the b-th
    // longest of them: a few dozen launches instead of one per member, whose
    // burst of pending launches at the start held up the other engine's graph
    std::vector<std::vector<int>> groups;
    std::vector<long long> keys;
    for (int k : b->order) {  // longest estimated solve first
        const ClusterShape &sh = b->shapes[k];
        const long long thr = (sh.threads + 127) / 128;
        long long mem = 8192;
        while (mem < (long long)sh.smem) mem *= 2;
        const long long key = (((long long)b->probs[k]->dtype * 64 + sh.G) * 16 + thr) * 64 +
                              (long long)log2((double)mem);
        const size_t q = (size_t)(std::find(keys.begin(), keys.end(), key) - keys.begin());
        if (q == keys.size()) {
            keys.push_back(key);
            groups.emplace_back();
        }
        groups[q].push_back(k);
    }
    std::vector<int> flat;
    for (auto &g : groups) flat.insert(flat.end(), g.begin(), g.end());
    ASYRK_CK(cudaMalloc((void **)&b->onchip_list, flat.size() * sizeof(int)));
    ASYRK_CK(cudaMemcpy(b->onchip_list, flat.data(), flat.size() * sizeof(int),
                        cudaMemcpyHostToDevice));
    size_t off = 0;
    for (auto &g : groups) {  // in the order of their longest members
        int threads = 0;
        size_t smem = 0;
        for (int k : g) {
            threads = std::max(threads, b->shapes[k].threads);
            smem = std::max(smem, b->shapes[k].smem);
        }
        const int k0 = g[0];
        int st = cluster_add_list_node(b->g_on, b->probs[k0]->dtype, b->shapes[k0].G, threads, smem,
                                       (int)g.size(), b->jobs, b->onchip_list + off);
        if (st != ASYRK_OK) return st;
        off += g.size();
    }
    ASYRK_CK(cudaGraphInstantiate(&b->exec_on, b->g_on, 0));
    return ASYRK_OK;
}

// Estimated time of one sweep of member k on its own CTA or cluster.
static double onchip_sweep_seconds(const asyrk_batch *b, int k)
{
    const asyrk_problem *p = b->probs[k];
    const ClusterShape &sh = b->shapes[k];
    const int64_t chunks = (p->max_len + 4 * sh.G - 1) / (4 * sh.G);
    const int64_t held = sh.G > 1 ? 2 : 1;  // chunks a lane keeps in registers
    const double per = ONCHIP_SECONDS_PER_PROJECTION *
                       (1.0 + ONCHIP_TAIL_CHUNK_FACTOR * (double)(chunks > held ? chunks - held : 0));
    return (double)p->m * per / sh.workers;
}

// Estimated time of one sweep of member k in the global engine when it has
// the GPU to itself: its Cor. 2 worker cap at the L2-bound projection time.
static double global_sweep_seconds(const asyrk_batch *b, int k)
{
    const asyrk_problem *p = b->probs[k];
    return (double)p->m * GLOBAL_SECONDS_PER_PROJECTION / (double)tau_cap_estimate(p->m, p->n);
}

// Which members the on-chip engine takes (b->on).  GLOBAL: none.  ONCHIP:
// all, EINVAL when one does not fit.  AUTO: those that fit, less the ones
// whose move to the global-iterate engine shortens the estimated batch time.
// Both engines run at once; per sweep, the on-chip part lasts as long as its
// longest member (or its thread-time over the GPU's threads, if longer), the
// global part as long as its longest member or its projections at the global
// rate, whichever is longer (constants measured, in cluster.cuh).
static int plan_members(asyrk_batch *b, int engine, int cluster_max, int max_workers, int update)
{
    b->on.assign(b->count, 0);
    if (engine == ASYRK_ENGINE_GLOBAL) return ASYRK_OK;
    if (update != ASYRK_UPDATE_ROW) {
        if (engine == ASYRK_ENGINE_ONCHIP)
            return set_error(ASYRK_EINVAL, "the on-chip engine runs the full-row update only");
        return ASYRK_OK;
    }
    b->shapes.assign(b->count, ClusterShape());
    std::set<long long> prepared;
    std::vector<int> cand;
    for (int k = 0; k < b->count; ++k) {
        asyrk_problem *p = b->probs[k];
        int st = cluster_shape(p, engine_subwarp(p, true), cluster_max, max_workers, &b->shapes[k]);
        if (st != ASYRK_OK) return st;
        const ClusterShape &sh = b->shapes[k];
        if (!sh.fits) {
            if (engine == ASYRK_ENGINE_ONCHIP)
                return set_error(ASYRK_EINVAL, "problem %d (m=%lld, n=%lld) does not fit the shared "
                                 "memory of a cluster", k, (long long)p->m, (long long)p->n);
            continue;
        }
        const long long key = ((long long)p->dtype * 64 + sh.G) * 2 + (sh.C > 1 ? 1 : 0);
        if (prepared.insert(key).second && (st = cluster_prepare(p->dtype, sh.G, sh.C)) != ASYRK_OK)
            return st;
        if ((st = cluster_check_schedulable(p->dtype, sh)) != ASYRK_OK) {
            if (engine == ASYRK_ENGINE_ONCHIP) return st;
            continue;
        }
        cand.push_back(k);
    }
    size_t first = 0;
    if (engine == ASYRK_ENGINE_AUTO && !cand.empty()) {
        std::vector<char> is_cand(b->count, 0);
        for (int k : cand) is_cand[k] = 1;
        double g_long = 0.0, g_proj = 0.0;  // the global part: longest member, projections
        for (int k = 0; k < b->count; ++k) {
            if (is_cand[k]) continue;
            g_long = std::max(g_long, global_sweep_seconds(b, k));
            g_proj += (double)b->probs[k]->m;
        }
        std::stable_sort(cand.begin(), cand.end(), [&](int u, int v) {
            return onchip_sweep_seconds(b, u) > onchip_sweep_seconds(b, v);
        });
        // thread-seconds per sweep of the on-chip members from position q on
        std::vector<double> area(cand.size() + 1, 0.0);
        for (size_t q = cand.size(); q-- > 0;)
            area[q] = area[q + 1] + onchip_sweep_seconds(b, cand[q]) *
                                        (double)b->shapes[cand[q]].threads * b->shapes[cand[q]].C;
        const double gpu_threads = THREADS_PER_SM * b->probs[0]->sm_count;
        auto on_time = [&](size_t q) {
            return q < cand.size() ? std::max(onchip_sweep_seconds(b, cand[q]), area[q] / gpu_threads)
                                   : 0.0;
        };
        auto glob_time = [&](double lng, double proj) {
            return std::max(lng, proj / GLOBAL_PROJECTIONS_PER_SECOND);
        };
        while (first < cand.size()) {
            const int k = cand[first];
            const double now = std::max(on_time(first), glob_time(g_long, g_proj));
            const double l2 = std::max(g_long, global_sweep_seconds(b, k));
            const double p2 = g_proj + (double)b->probs[k]->m;
            if (std::max(on_time(first + 1), glob_time(l2, p2)) >= now) break;
            g_long = l2;
            g_proj = p2;
            ++first;
        }
    }
    for (size_t q = first; q < cand.size(); ++q) b->on[cand[q]] = 1;
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
    if (o.engine < ASYRK_ENGINE_AUTO || o.engine > ASYRK_ENGINE_ONCHIP)
        return set_error(ASYRK_EINVAL, "unknown engine %d", (int)o.engine);
    if (o.cluster_max != 0 && o.cluster_max != 1 && o.cluster_max != 2 && o.cluster_max != 4 &&
        o.cluster_max != 8)
        return set_error(ASYRK_EINVAL, "cluster_max must be 0, 1, 2, 4 or 8");
    if (o.workers < 0) return set_error(ASYRK_EINVAL, "workers < 0");
    if (o.partition < -1) return set_error(ASYRK_EINVAL, "partition must be >= -1");
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
        // the plan splits the warps in proportion to this.  A worker's
        // projection takes about 3.6 us + 0.63 us per entry a lane handles
        // (L/G of them; measured per slot on the 256-system workload), and a
        // sweep lasts m / workers = m G / (32 warps) projections of it, so
        // equal sweeps want warps in proportion to m (5.7 G + L)
        D.work = (double)p->m * (6.0 * (double)G) + (double)p->nnz;
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
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev_done[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev_done[1]);
    if (e != cudaSuccess) return fail(cuda_fail(e, "batch allocation", __FILE__, __LINE__));
    for (int k = 0; k < count; ++k) {
        b->h[k].x = b->x + b->xoff[k];
        b->h[k].x64 = b->x64 + b->xoff[k];
        b->h[k].busy = b->busy + busy_off[k];
    }
    if ((st = plan_members(b, o.engine, o.cluster_max, o.workers, o.update)) != ASYRK_OK)
        return fail(st);
    for (int k = 0; k < count; ++k) (b->on[k] ? b->n_on : b->n_glob) += 1;
    if (b->n_on > 0) {
        for (int k = 0; k < count; ++k)
            if (b->on[k]) b->order.push_back(k);
        std::stable_sort(b->order.begin(), b->order.end(), [&](int u, int v) {
            return onchip_sweep_seconds(b, u) > onchip_sweep_seconds(b, v);
        });
        b->hj.assign(count, ClusterJob());
        for (int k : b->order) {
            asyrk_problem *p = problems[k];
            const ClusterShape &sh = b->shapes[k];
            ClusterJob &J = b->hj[k];
            memset(&J, 0, sizeof J);
            J.rec = p->rec;
            J.col = p->col;
            J.val = p->val;
            J.x64 = b->x64 + b->xoff[k];
            J.x32 = b->x + b->xoff[k];
            J.key = b->h[k].key;
            J.m = (unsigned)p->m;
            J.n = (unsigned)p->n;
            J.uniform = p->uniform;
            J.sampling = o.sampling;
            J.shuf_h = b->h[k].shuf_h;
            J.excl = b->excl ? 1 : 0;
            J.workers = sh.workers;
            J.lc = sh.lc;
            J.nper = sh.nper;
            J.nper_pad = sh.nper_pad;
            J.bper = sh.bper;
        }
        e = cudaMalloc((void **)&b->jobs, count * sizeof(ClusterJob));
        if (e == cudaSuccess && b->n_glob > 0)
            e = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking);
        if (e == cudaSuccess && b->n_glob > 0)
            e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
        if (e == cudaSuccess && b->n_glob > 0)
            e = cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming);
        if (e != cudaSuccess) return fail(cuda_fail(e, "on-chip batch set-up", __FILE__, __LINE__));
    }
    if (b->n_glob > 0 && b->n_on > 0 && b->graph && o.partition >= 0) {
        // SMs for the on-chip engine: its members' thread-time per sweep within
        // 1/2.5 of its longest member's sweep (one CTA each; clusters need
        // co-scheduled SMs and keep the whole GPU)
        double longest = 0.0, area = 0.0;
        bool single = true;
        for (int k = 0; k < count; ++k) {
            if (!b->on[k]) continue;
            const double t = onchip_sweep_seconds(b, k);
            longest = std::max(longest, t);
            area += t * (double)b->shapes[k].threads;
            single = single && b->shapes[k].C == 1;
        }
        int on_sms = o.partition > 0
                         ? o.partition
                         : (int)ceil(2.5 * area / (THREADS_PER_SM * (longest > 0.0 ? longest : 1.0)));
        on_sms = std::max(8, std::min(on_sms, sms - 8));
        if (single && sm_partition_create(dev, sms - on_sms, &b->split)) {
            b->resident_warps_glob =
                std::max(8, (int)((long long)b->resident_warps * b->split.sms[0] / sms));
            if (cudaEventCreateWithFlags(&b->ev_on_join, cudaEventDisableTiming) != cudaSuccess)
                return fail(cuda_fail(cudaGetLastError(), "batch event", __FILE__, __LINE__));
        }
    }
    if (b->n_on > 0 && b->graph && (st = build_onchip_graph(b, b->split.ctx[1] != nullptr)) != ASYRK_OK)
        return fail(st);
    if (b->n_glob > 0 && b->graph && (st = build_graph(b)) != ASYRK_OK) return fail(st);
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
    // on-chip members sit out of the global engine's table; their jobs get the
    // solve's parameters
    for (int k = 0; k < b->count; ++k) {
        if (!b->on[k]) continue;
        SysDesc &D = b->h[k];
        D.active = 0;
        ClusterJob &J = b->hj[k];
        J.gamma = D.gamma;
        J.tol = D.tol;
        J.max_sweeps = max_sweeps;
        J.j0 = D.j;
        J.xt = D.xt;
        J.bnorm = b->probs[k]->bnorm;
        J.meas = J.meas0 = -1.0;
        J.sweeps = 0;
        J.skipped = 0;
        J.status = ASYRK_NOT_CONVERGED;
    }
    int st = launch_batch_convert(b->x64, b->x, b->n_total, true, s);
    if (st != ASYRK_OK) return st;
    ASYRK_CK(cudaMemcpyAsync(b->d, b->h.data(), b->count * sizeof(SysDesc), cudaMemcpyHostToDevice, s));
    if (b->n_on > 0)
        ASYRK_CK(cudaMemcpyAsync(b->jobs, b->hj.data(), b->count * sizeof(ClusterJob),
                                 cudaMemcpyHostToDevice, s));
    const int max_iter = (int)(max_sweeps < 0x3ffffffe ? max_sweeps + 1 : 0x3fffffff);
    b->h_ints[1] = 0;
    b->h_ints[2] = 0;
    b->h_ints[3] = max_iter;
    ASYRK_CK(cudaMemcpyAsync(b->d_iter, b->h_ints + 2, 2 * sizeof(int), cudaMemcpyHostToDevice, s));
    int64_t launches = 2;  // the two conversions
    int64_t iters = 0;
    ASYRK_CK(cudaEventRecord(b->ev[0], s));
    // the global engine's members: on a second stream when the on-chip engine
    // runs at the same time (graph form), else on the batch's stream
    const bool both = b->n_on > 0 && b->n_glob > 0 && b->graph;
    cudaStream_t gs = both ? (b->split.stream[0] ? b->split.stream[0] : b->side) : s;
    cudaStream_t os = (both && b->split.stream[1]) ? b->split.stream[1] : s;
    if (b->n_glob > 0) {
        if (gs != s) {
            ASYRK_CK(cudaEventRecord(b->ev_fork, s));
            ASYRK_CK(cudaStreamWaitEvent(gs, b->ev_fork, 0));
        }
        if ((st = launch_batch_measure(b->d, b->count, b->total_chunks, b->part, gs)) != ASYRK_OK)
            return st;
        launches += 1;
        if (b->graph) {
            ASYRK_CK(cudaGraphLaunch(b->exec, gs));
            ASYRK_CK(cudaMemcpyAsync(b->h_ints + 1, b->d_iter, sizeof(int), cudaMemcpyDeviceToHost, gs));
        } else {
            for (int it = 0; it < max_iter; ++it) {
                if ((st = launch_batch_iteration(b->d, b->count, b->total_chunks, b->part,
                                                 b->resident_warps, b->excl, b->d_active,
                                                 b->d_iter, false, 0ull, gs)) != ASYRK_OK)
                    return st;
                ASYRK_CK(cudaMemcpyAsync(b->h_ints, b->d_active, sizeof(int), cudaMemcpyDeviceToHost, gs));
                ASYRK_CK(cudaStreamSynchronize(gs));
                ++b->h_ints[1];
                if (b->h_ints[0] == 0) break;
            }
        }
        ASYRK_CK(cudaEventRecord(b->ev_done[0], gs));
        if (gs != s) ASYRK_CK(cudaEventRecord(b->ev_join, gs));
    }
    if (b->n_on > 0) {
        if (os != s) {
            ASYRK_CK(cudaEventRecord(b->ev_fork, s));
            ASYRK_CK(cudaStreamWaitEvent(os, b->ev_fork, 0));
        }
        if (b->graph) {
            ASYRK_CK(cudaGraphLaunch(b->exec_on, os));
        } else {
            for (int k : b->order)
                if ((st = cluster_launch(b->probs[k]->dtype, b->shapes[k], b->jobs, k, s)) != ASYRK_OK)
                    return st;
        }
        launches += b->n_on;
        ASYRK_CK(cudaEventRecord(b->ev_done[1], os));
        if (os != s) {
            ASYRK_CK(cudaEventRecord(b->ev_on_join, os));
            ASYRK_CK(cudaStreamWaitEvent(s, b->ev_on_join, 0));
        }
        ASYRK_CK(cudaMemcpyAsync(b->hj.data(), b->jobs, b->count * sizeof(ClusterJob),
                                 cudaMemcpyDeviceToHost, s));
    }
    if (b->n_glob > 0 && gs != s) ASYRK_CK(cudaStreamWaitEvent(s, b->ev_join, 0));
    ASYRK_CK(cudaEventRecord(b->ev[1], s));
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
    if (b->n_glob > 0) {
        iters = b->h_ints[1];
        launches += 4 * iters;
    }
    for (int k = 0; k < b->count; ++k) {  // the on-chip members' outcomes
        if (!b->on[k]) continue;
        const ClusterJob &J = b->hj[k];
        SysDesc &D = b->h[k];
        D.sweeps = J.sweeps;
        D.status = J.status;
        D.meas = J.meas;
        D.meas0 = J.meas0;
        D.j = J.j0 + (unsigned long long)J.sweeps * (unsigned long long)J.m;
        D.skipped = J.skipped;
        if (J.sweeps > iters) iters = J.sweeps;
    }
    float ms = 0.f, part_ms[2] = {0.f, 0.f};
    ASYRK_CK(cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]));
    for (int q = 0; q < 2; ++q) {
        if ((q == 0 ? b->n_glob : b->n_on) == 0) continue;
        if (cudaEventElapsedTime(&part_ms[q], b->ev[0], b->ev_done[q]) != cudaSuccess) {
            part_ms[q] = -1.f;  // a timing the driver does not give is reported as -1
            (void)cudaGetLastError();
        }
    }
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
            I.workers = b->on[k] ? b->shapes[k].workers : D.first_nwarps * (32 / D.G);
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
        binfo->engine = (b->n_glob > 0 ? ASYRK_ENGINE_GLOBAL : 0) | (b->n_on > 0 ? ASYRK_ENGINE_ONCHIP : 0);
        binfo->onchip_members = b->n_on;
        binfo->global_sms = b->split.sms[0];
        binfo->global_ms = part_ms[0];
        binfo->onchip_ms = part_ms[1];
        binfo->reserved = 0;
    }
    return worst;
}
