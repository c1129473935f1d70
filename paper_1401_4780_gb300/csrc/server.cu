// server.cu -- asyrk_server_*: continuous batching of solve requests.
//
// Requests name a problem that is already resident (asyrk_create) and bring
// their own x0 (and optionally x*), step length, tolerance and mode.  An engine
// thread owns the GPU side and repeats:
//   admit    queued requests enter free slots while the device-memory budget
//            allows (a slot's iterate, staging, claim bits and refinement
//            residual come from a native arena; a problem's own bytes count
//            once while any request uses it);
//   iterate  one engine step over all occupied slots (batch.cuh: plan,
//            project, check, and the outer step of refinement slots), so the
//            row projections of every admitted request share one persistent
//            kernel launch;
//   harvest  finished slots copy their x back, free their memory and wake
//            the request's waiter; the next admission can take the slot.
// A request whose problem fits a CTA's shared memory (cluster.cu) skips the
// shared engine step: it takes an on-chip slot, its whole solve (plain or
// refined) is one CTA launch on the slot's own stream, and the engine thread
// harvests it when the launch's event has completed; such requests may pass
// queued requests that wait for memory or for a slot of the shared step.
// Every request has its own Philox stream (the ticket), so one problem can
// serve several requests at once.  The device never waits on the host: every
// wait is host-side and has a time limit.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "batch.cuh"
#include "cluster.cuh"
#include "partition.cuh"

namespace asyrk {

// ---------------------------------------------------------------------------
// Device arena: chunks from cudaMalloc, carved first-fit into 256-byte aligned
// blocks; a freed block coalesces with free neighbours.
// ---------------------------------------------------------------------------
class Arena {
  public:
    explicit Arena(size_t limit) : limit_(limit) {}
    ~Arena()
    {
        for (auto &c : chunks_) cudaFree(c.base);
    }
    Arena(const Arena &) = delete;
    Arena &operator=(const Arena &) = delete;

    // nullptr when the limit would be exceeded or cudaMalloc fails
    void *alloc(size_t bytes)
    {
        bytes = round(bytes);
        for (auto &c : chunks_) {
            for (auto it = c.free.begin(); it != c.free.end(); ++it) {
                if (it->second < bytes) continue;
                const size_t off = it->first, len = it->second;
                c.free.erase(it);
                if (len > bytes) c.free[off + bytes] = len - bytes;
                return c.base + off;
            }
        }
        size_t sz = bytes > kChunk ? bytes : kChunk;
        if (reserved_ + sz > limit_) sz = bytes;
        if (reserved_ + sz > limit_) return nullptr;
        Chunk c;
        if (cudaMalloc((void **)&c.base, sz) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        c.size = sz;
        if (sz > bytes) c.free[bytes] = sz - bytes;
        reserved_ += sz;
        chunks_.push_back(std::move(c));
        return chunks_.back().base;
    }

    void release(void *p, size_t bytes)
    {
        if (!p) return;
        bytes = round(bytes);
        char *q = static_cast<char *>(p);
        for (auto &c : chunks_) {
            if (q < c.base || q >= c.base + c.size) continue;
            size_t off = (size_t)(q - c.base), len = bytes;
            auto next = c.free.lower_bound(off);
            if (next != c.free.end() && off + len == next->first) {
                len += next->second;
                next = c.free.erase(next);
            }
            if (next != c.free.begin()) {
                auto prev = std::prev(next);
                if (prev->first + prev->second == off) {
                    off = prev->first;
                    len += prev->second;
                    c.free.erase(prev);
                }
            }
            c.free[off] = len;
            return;
        }
    }

    size_t reserved() const { return reserved_; }

  private:
    static constexpr size_t kChunk = (size_t)256 << 20;
    static size_t round(size_t b) { return (b + 255) & ~(size_t)255; }
    struct Chunk {
        char *base = nullptr;
        size_t size = 0;
        std::map<size_t, size_t> free;  // offset -> length
    };
    std::vector<Chunk> chunks_;
    size_t limit_;
    size_t reserved_ = 0;
};

struct Request {
    uint64_t ticket = 0;
    asyrk_problem *p = nullptr;
    std::vector<double> x0, xt, result;
    double gamma = 1.0, tol = 0.0;
    int mode = ASYRK_MODE_ASYNC;
    int64_t max_sweeps = 0;
    double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
    int status = ASYRK_NOT_CONVERGED;
    bool done = false, cancelled = false;
    int slot = -1;
    size_t slot_bytes = 0;
    bool onchip = false;   // solved by one CTA (ocshape) instead of the shared engine step
    ClusterShape ocshape;
    long long demand = 0;  // warps the shared step would give it alone (its Cor. 2 cap)
    asyrk_solve_info info;
};

struct SlotMem {
    float *x = nullptr;
    double *x64 = nullptr, *xt = nullptr;
    unsigned *busy = nullptr;
    float *r32 = nullptr;
    size_t bx = 0, bx64 = 0, bxt = 0, bbusy = 0, br32 = 0;
};

static double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

}  // namespace asyrk

using namespace asyrk;

struct asyrk_server {
    int max_slots = 0;
    size_t budget = 0;
    bool excl = true;
    int device = 0;
    int resident_warps = 0;
    double inner_tol = 1e-3;
    int64_t max_inner = 60;
    double admit_load = 1.0;   // <= 0: admission bounded by slots and memory only
    int max_active_shared = 0;
    // the shared step (group 0, stream s) and the on-chip requests (group 1) on
    // disjoint SMs, when split
    SmPartition split;
    int step_warps = 0;        // the step's resident warps on its SMs (split only)
    cudaStream_t s = nullptr;
    SysDesc *d = nullptr;
    std::vector<SysDesc> h;
    std::vector<Request *> slot_req;
    std::vector<SlotMem> slot_mem;
    double *part = nullptr;
    int part_cap = 0;
    Arena *arena = nullptr;
    size_t used = 0;
    std::map<asyrk_problem *, int> problem_refs;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;      // requests for the shared engine step
    std::deque<Request *> oc_queue;   // requests solved on-chip
    std::unordered_map<uint64_t, Request *> reqs;
    uint64_t next_ticket = 1;
    bool stop = false;
    int fatal = ASYRK_OK;
    std::thread th;
    std::thread oc_th;                // admits and harvests the on-chip requests
    std::condition_variable cv_oc;

    int64_t submitted = 0, completed = 0, iterations = 0, launches = 0, max_active = 0;

    // on-chip slots: one CTA launch per request, each slot with its own stream
    bool onchip = true;
    int oc_slots = 0;
    std::vector<Request *> oc_req;
    std::vector<SlotMem> oc_mem;
    std::vector<ClusterJob> oc_hj;
    ClusterJob *oc_jobs = nullptr;
    std::vector<cudaStream_t> oc_stream;
    std::vector<cudaEvent_t> oc_ev;
    std::vector<float> oc_x32;          // staging of a plain solve's FP32 x
    std::vector<long long> oc_prepared;  // (dtype, G) kernels given their shared memory
    int64_t oc_completed = 0;
};

static size_t request_bytes(const asyrk_problem *p, bool has_xt, int mode)
{
    size_t b = (size_t)p->n * (4 + 8) + (size_t)((p->m + 31) / 32) * 4;
    if (has_xt) b += (size_t)p->n * 8;
    if (mode == ASYRK_MODE_REFINE) b += (size_t)p->m * 4;
    return b + 5 * 256;
}

static void free_slot_mem(asyrk_server *sv, int k)
{
    SlotMem &M = sv->slot_mem[k];
    sv->arena->release(M.x, M.bx);
    sv->arena->release(M.x64, M.bx64);
    sv->arena->release(M.xt, M.bxt);
    sv->arena->release(M.busy, M.bbusy);
    sv->arena->release(M.r32, M.br32);
    M = SlotMem();
}

// complete a request, with sv->mu held
static void finish_locked(asyrk_server *sv, Request *r, int status)
{
    r->status = status;
    r->info.status = status;
    r->t_done = now_s();
    r->info.seconds = r->t_done - r->t_submit;
    r->done = true;
    sv->completed += 1;
    sv->cv_done.notify_all();
}

// admit request r into slot k (engine thread, sv->mu held); false: no memory now
static bool admit_locked(asyrk_server *sv, Request *r, int k)
{
    asyrk_problem *p = r->p;
    const bool has_xt = !r->xt.empty();
    const bool refine = r->mode == ASYRK_MODE_REFINE;
    const size_t need = r->slot_bytes + (sv->problem_refs.count(p) ? 0 : (size_t)p->dev_bytes);
    if (sv->used + need > sv->budget) return false;
    SlotMem M;
    M.bx = (size_t)p->n * 4;
    M.bx64 = (size_t)p->n * 8;
    M.bbusy = (size_t)((p->m + 31) / 32) * 4;
    M.bxt = has_xt ? (size_t)p->n * 8 : 0;
    M.br32 = refine ? (size_t)p->m * 4 : 0;
    M.x = (float *)sv->arena->alloc(M.bx);
    M.x64 = (double *)sv->arena->alloc(M.bx64);
    M.busy = (unsigned *)sv->arena->alloc(M.bbusy);
    if (has_xt) M.xt = (double *)sv->arena->alloc(M.bxt);
    if (refine) M.r32 = (float *)sv->arena->alloc(M.br32);
    sv->slot_mem[k] = M;
    if (!M.x || !M.x64 || !M.busy || (has_xt && !M.xt) || (refine && !M.r32)) {
        free_slot_mem(sv, k);
        return false;
    }
    sv->used += need;
    sv->problem_refs[p] += 1;
    // x0 -> x64; plain slots iterate on x (FP32); refinement slots keep x64 as
    // the iterate and x as the FP32 correction, starting at zero
    cudaMemcpyAsync(M.x64, r->x0.data(), M.bx64, cudaMemcpyHostToDevice, sv->s);
    if (has_xt) cudaMemcpyAsync(M.xt, r->xt.data(), M.bxt, cudaMemcpyHostToDevice, sv->s);
    cudaMemsetAsync(M.busy, 0, M.bbusy, sv->s);
    if (refine) {
        cudaMemsetAsync(M.x, 0, M.bx, sv->s);
    } else {
        launch_batch_convert(M.x64, M.x, p->n, true, sv->s);
        sv->launches += 1;
    }
    SysDesc &D = sv->h[k];
    memset(&D, 0, sizeof D);
    const int G = engine_subwarp(p, false);
    const long long capw = tau_cap_estimate(p->m, p->n);
    const long long cw = (capw * G + 31) / 32;
    D.G = G;
    D.cap_warps = (int)(cw < 1 ? 1 : cw > 0x7fffffff ? 0x7fffffff : cw);
    D.rec = p->rec;
    D.col = p->col;
    D.val = p->val;
    D.b64 = p->b64;
    D.x = M.x;
    D.x64 = M.x64;
    D.xt = M.xt;
    D.busy = M.busy;
    D.r32 = M.r32;
    D.bvec = refine ? M.r32 : nullptr;
    D.m = (unsigned)p->m;
    D.n = (unsigned)p->n;
    D.dtype = p->dtype;
    D.uniform = p->uniform;
    D.work = (double)p->nnz;
    D.key = make_uint2((unsigned)p->seed, (unsigned)(p->seed >> 32));
    D.stream_id = (unsigned)r->ticket;  // each request draws its own row sequence
    D.j = 0;
    D.gamma = (float)r->gamma;
    D.tol = r->tol;
    D.max_sweeps = r->max_sweeps;
    D.active = 1;
    D.status = ASYRK_NOT_CONVERGED;
    D.meas = -1.0;
    D.meas0 = -1.0;
    double xtn = 0.0;
    for (double v : r->xt) xtn += v * v;
    xtn = sqrt(xtn);
    const double bn = p->bnorm > 0.0 ? p->bnorm : 1.0;
    D.mode = refine ? SLOT_REFINE : SLOT_PLAIN;
    D.phase = refine ? 1 : 0;  // refinement starts with an outer step: r = b - A x0
    D.ref = has_xt ? (xtn > 0.0 ? xtn : 1.0) : bn;
    D.outer_ref = D.ref;
    D.inner_tol = sv->inner_tol;
    D.inner_goal = sv->inner_tol;
    D.max_inner = sv->max_inner;
    D.max_k = 32;  // short sweeps run several per engine step
    D.sampling = ASYRK_SAMPLE_WEIGHTED;
    D.update = ASYRK_UPDATE_ROW;
    D.shuf_h = shuffle_half_bits(p->m);
    sv->slot_req[k] = r;
    r->slot = k;
    r->t_admit = now_s();
    return true;
}

static void release_slot_locked(asyrk_server *sv, int k)
{
    Request *r = sv->slot_req[k];
    asyrk_problem *p = r->p;
    free_slot_mem(sv, k);
    size_t give = r->slot_bytes;
    if (--sv->problem_refs[p] == 0) {
        sv->problem_refs.erase(p);
        give += (size_t)p->dev_bytes;
    }
    sv->used -= give;
    sv->slot_req[k] = nullptr;
    memset(&sv->h[k], 0, sizeof(SysDesc));
    r->slot = -1;
}

// admit request r into on-chip slot k and launch its solve (engine thread,
// sv->mu held); false: no memory now
static bool admit_onchip_locked(asyrk_server *sv, Request *r, int k)
{
    asyrk_problem *p = r->p;
    const bool has_xt = !r->xt.empty();
    const bool refine = r->mode == ASYRK_MODE_REFINE;
    const size_t need = r->slot_bytes + (sv->problem_refs.count(p) ? 0 : (size_t)p->dev_bytes);
    if (sv->used + need > sv->budget) return false;
    SlotMem M;
    M.bx = (size_t)p->n * 4;
    M.bx64 = (size_t)p->n * 8;
    M.bxt = has_xt ? (size_t)p->n * 8 : 0;
    M.br32 = refine ? (size_t)p->m * 4 : 0;
    M.x = (float *)sv->arena->alloc(M.bx);
    M.x64 = (double *)sv->arena->alloc(M.bx64);
    if (has_xt) M.xt = (double *)sv->arena->alloc(M.bxt);
    if (refine) M.r32 = (float *)sv->arena->alloc(M.br32);
    sv->oc_mem[k] = M;
    if (!M.x || !M.x64 || (has_xt && !M.xt) || (refine && !M.r32)) {
        SlotMem &F = sv->oc_mem[k];
        sv->arena->release(F.x, F.bx);
        sv->arena->release(F.x64, F.bx64);
        sv->arena->release(F.xt, F.bxt);
        sv->arena->release(F.r32, F.br32);
        F = SlotMem();
        return false;
    }
    sv->used += need;
    sv->problem_refs[p] += 1;
    const ClusterShape &sh = r->ocshape;
    ClusterJob &J = sv->oc_hj[k];
    memset(&J, 0, sizeof J);
    J.rec = p->rec;
    J.col = p->col;
    J.val = p->val;
    J.x64 = M.x64;
    J.x32 = M.x;
    J.xt = M.xt;
    J.b64 = p->b64;
    J.r32 = M.r32;
    J.key = make_uint2((unsigned)p->seed, (unsigned)(p->seed >> 32));
    J.m = (unsigned)p->m;
    J.n = (unsigned)p->n;
    J.stream_id = (unsigned)r->ticket;  // each request draws its own row sequence
    J.uniform = p->uniform;
    J.sampling = ASYRK_SAMPLE_WEIGHTED;
    J.shuf_h = shuffle_half_bits(p->m);
    J.excl = sv->excl ? 1 : 0;
    J.workers = sh.workers;
    J.lc = sh.lc;
    J.nper = sh.nper;
    J.nper_pad = sh.nper_pad;
    J.bper = sh.bper;
    J.gamma = (float)r->gamma;
    J.refine = refine ? 1 : 0;
    J.max_inner = sv->max_inner;
    J.inner_tol = sv->inner_tol;
    J.j0 = 0;
    J.max_sweeps = r->max_sweeps;
    J.tol = r->tol;
    J.bnorm = p->bnorm;
    J.meas = J.meas0 = -1.0;
    J.status = ASYRK_NOT_CONVERGED;
    // the slot's stream is idle (its previous request was harvested), so these
    // copies from pageable memory do not wait on other work
    cudaStream_t st = sv->oc_stream[k];
    cudaMemcpyAsync(M.x64, r->x0.data(), M.bx64, cudaMemcpyHostToDevice, st);
    if (has_xt) cudaMemcpyAsync(M.xt, r->xt.data(), M.bxt, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(sv->oc_jobs + k, &J, sizeof J, cudaMemcpyHostToDevice, st);
    int rc = cluster_launch(p->dtype, sh, sv->oc_jobs, k, st);
    if (rc == ASYRK_OK && cudaEventRecord(sv->oc_ev[k], st) != cudaSuccess) rc = ASYRK_ECUDA;
    sv->launches += 1;
    sv->oc_req[k] = r;
    r->slot = k;
    r->t_admit = now_s();
    if (rc != ASYRK_OK) sv->fatal = rc;  // the engine loop stops the server
    return true;
}

static void release_onchip_locked(asyrk_server *sv, int k)
{
    Request *r = sv->oc_req[k];
    asyrk_problem *p = r->p;
    SlotMem &M = sv->oc_mem[k];
    sv->arena->release(M.x, M.bx);
    sv->arena->release(M.x64, M.bx64);
    sv->arena->release(M.xt, M.bxt);
    sv->arena->release(M.r32, M.br32);
    M = SlotMem();
    size_t give = r->slot_bytes;
    if (--sv->problem_refs[p] == 0) {
        sv->problem_refs.erase(p);
        give += (size_t)p->dev_bytes;
    }
    sv->used -= give;
    sv->oc_req[k] = nullptr;
    r->slot = -1;
}

// complete the on-chip requests whose launch has finished; *any: one did
static int harvest_onchip(asyrk_server *sv, std::unique_lock<std::mutex> &lk, bool *any)
{
    *any = false;
    for (int k = 0; k < sv->oc_slots; ++k) {
        Request *r = sv->oc_req[k];
        if (!r) continue;
        const cudaError_t q = cudaEventQuery(sv->oc_ev[k]);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) return cuda_fail(q, "on-chip request", __FILE__, __LINE__);
        const SlotMem M = sv->oc_mem[k];
        const unsigned n = (unsigned)r->p->n;
        const bool refine = r->mode == ASYRK_MODE_REFINE;
        lk.unlock();
        // the launch has finished: these copies on the slot's stream run at once
        cudaStream_t cs = sv->oc_stream[k];
        ClusterJob J;
        r->result.resize(n);
        cudaError_t e = cudaMemcpyAsync(&J, sv->oc_jobs + k, sizeof J, cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess && refine) {
            e = cudaMemcpyAsync(r->result.data(), M.x64, (size_t)n * 8, cudaMemcpyDeviceToHost, cs);
        } else if (e == cudaSuccess) {
            sv->oc_x32.resize(n);
            e = cudaMemcpyAsync(sv->oc_x32.data(), M.x, (size_t)n * 4, cudaMemcpyDeviceToHost, cs);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
        if (e == cudaSuccess && !refine)
            for (unsigned t = 0; t < n; ++t) r->result[t] = (double)sv->oc_x32[t];
        lk.lock();
        if (e != cudaSuccess) return cuda_fail(e, "on-chip harvest", __FILE__, __LINE__);
        asyrk_solve_info &I = r->info;
        memset(&I, 0, sizeof I);
        I.workers = r->ocshape.workers;
        I.subwarp = r->ocshape.G;
        I.refine_steps = J.outer_steps;
        I.sweeps = J.sweeps;
        I.projections = J.sweeps * (int64_t)J.m;
        I.skipped = (int64_t)J.skipped;
        I.rel_err = r->xt.empty() ? -1.0 : J.meas;
        I.rel_res = refine && r->p->bnorm > 0.0 ? sqrt(J.res2) / r->p->bnorm : -1.0;
        I.j_end = (uint64_t)J.sweeps * J.m;
        const int status = r->cancelled ? ASYRK_ECANCELED : J.status;
        release_onchip_locked(sv, k);
        finish_locked(sv, r, status);
        sv->oc_completed += 1;
        *any = true;
    }
    return ASYRK_OK;
}

// complete every shared-step request (in a slot or queued) with `status`
static void fail_shared_locked(asyrk_server *sv, int status)
{
    for (int k = 0; k < sv->max_slots; ++k) {
        if (!sv->slot_req[k]) continue;
        Request *r = sv->slot_req[k];
        release_slot_locked(sv, k);
        finish_locked(sv, r, status);
    }
    while (!sv->queue.empty()) {
        Request *r = sv->queue.front();
        sv->queue.pop_front();
        finish_locked(sv, r, status);
    }
}

// complete every on-chip request with `status`; launches in flight run to
// their end first (their memory is released after them)
static void fail_onchip_locked(asyrk_server *sv, int status)
{
    for (int k = 0; k < sv->oc_slots; ++k) {
        if (!sv->oc_req[k]) continue;
        cudaStreamSynchronize(sv->oc_stream[k]);
        Request *r = sv->oc_req[k];
        release_onchip_locked(sv, k);
        finish_locked(sv, r, status);
    }
    while (!sv->oc_queue.empty()) {
        Request *r = sv->oc_queue.front();
        sv->oc_queue.pop_front();
        finish_locked(sv, r, status);
    }
}

// one engine step over the occupied slots, GPU work done without the lock
static int engine_step(asyrk_server *sv, std::unique_lock<std::mutex> &lk, std::vector<int> &done)
{
    // the descriptors up to the last occupied slot are all the step reads
    int hi = 0;
    for (int k = 0; k < sv->max_slots; ++k)
        if (sv->slot_req[k]) hi = k + 1;
    int chunks = 0;
    for (int k = 0; k < hi; ++k) {
        SysDesc &D = sv->h[k];
        D.chunk0 = chunks;
        if (!sv->slot_req[k]) {
            D.nchunks = 0;
            continue;
        }
        const int64_t ce = ((int64_t)D.n + BATCH_ERR_CHUNK - 1) / BATCH_ERR_CHUNK;
        const int64_t cr = ((int64_t)D.m + BATCH_ROW_CHUNK - 1) / BATCH_ROW_CHUNK;
        D.nchunks = (int)(ce > cr ? ce : cr);
        chunks += D.nchunks;
        if (sv->slot_req[k]->cancelled) D.active = 0;
    }
    if (chunks > sv->part_cap) {
        cudaFree(sv->part);
        sv->part = nullptr;
        sv->part_cap = 0;
        ASYRK_CK(cudaMalloc((void **)&sv->part, 2 * (size_t)chunks * sizeof(double)));
        sv->part_cap = chunks;
    }
    // while on-chip launches are in flight the step takes three quarters of the
    // resident warps, so that none of its blocks waits for an SM that an
    // on-chip CTA occupies (a step lasts as long as its last block), and
    // on-chip requests that arrive during the step find room at once
    int oc = 0;
    for (int k = 0; k < sv->oc_slots; ++k) oc += sv->oc_req[k] ? 1 : 0;
    const int warps = sv->step_warps > 0 ? sv->step_warps
                      : oc > 0           ? sv->resident_warps / 4 * 3
                                         : sv->resident_warps;
    lk.unlock();
    int st = ASYRK_OK;
    cudaError_t e = cudaMemcpyAsync(sv->d, sv->h.data(), hi * sizeof(SysDesc),
                                    cudaMemcpyHostToDevice, sv->s);
    if (e == cudaSuccess)
        st = launch_engine_step(sv->d, hi, chunks, sv->part, warps, sv->excl, true, sv->s);
    if (e == cudaSuccess && st == ASYRK_OK)
        e = cudaMemcpyAsync(sv->h.data(), sv->d, hi * sizeof(SysDesc), cudaMemcpyDeviceToHost,
                            sv->s);
    if (e == cudaSuccess && st == ASYRK_OK) e = cudaStreamSynchronize(sv->s);
    lk.lock();
    if (e != cudaSuccess) return cuda_fail(e, "server step", __FILE__, __LINE__);
    if (st != ASYRK_OK) return st;
    sv->iterations += 1;
    sv->launches += 5;
    done.clear();
    for (int k = 0; k < hi; ++k)
        if (sv->slot_req[k] && !sv->h[k].active) done.push_back(k);
    return ASYRK_OK;
}

// copy finished slots' x back and complete their requests
static int harvest(asyrk_server *sv, std::unique_lock<std::mutex> &lk, const std::vector<int> &done)
{
    if (done.empty()) return ASYRK_OK;
    lk.unlock();
    cudaError_t e = cudaSuccess;
    for (int k : done) {
        Request *r = sv->slot_req[k];
        const SysDesc &D = sv->h[k];
        r->result.resize(D.n);
        if (D.mode == SLOT_PLAIN) {
            if (launch_batch_convert(D.x64, D.x, D.n, false, sv->s) != ASYRK_OK) e = cudaErrorUnknown;
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(r->result.data(), D.x64, (size_t)D.n * sizeof(double),
                                cudaMemcpyDeviceToHost, sv->s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(sv->s);
    lk.lock();
    if (e != cudaSuccess) return cuda_fail(e, "server harvest", __FILE__, __LINE__);
    for (int k : done) {
        Request *r = sv->slot_req[k];
        const SysDesc &D = sv->h[k];
        asyrk_solve_info &I = r->info;
        memset(&I, 0, sizeof I);
        I.workers = D.first_nwarps * (32 / (D.G > 0 ? D.G : 32));
        I.subwarp = D.G;
        I.refine_steps = D.outer_steps;
        I.sweeps = D.sweeps;
        I.projections = D.sweeps * (int64_t)D.m;
        I.skipped = (int64_t)D.skipped;
        I.rel_err = D.xt ? D.meas : -1.0;
        I.rel_res = D.mode == SLOT_REFINE && r->p->bnorm > 0.0 ? sqrt(D.res2) / r->p->bnorm : -1.0;
        I.j_end = D.j;
        const int status = r->cancelled ? ASYRK_ECANCELED : D.status;
        release_slot_locked(sv, k);
        finish_locked(sv, r, status);
    }
    sv->launches += (int64_t)done.size();
    return ASYRK_OK;
}

static void engine_loop(asyrk_server *sv)
{
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    std::vector<int> done;
    for (;;) {
        // admission: FIFO into free slots while memory allows and while the
        // warp demands of the requests in the step stay within admit_load x the
        // resident warps.  Past that point another request would only split the
        // warps further: every request in the step would run with fewer, more
        // latency-bound workers and all of them would finish late, so the rest
        // wait in the queue (one request is always admitted).
        long long demand = 0;
        int in_step = 0;
        for (int k = 0; k < sv->max_slots; ++k)
            if (sv->slot_req[k]) {
                demand += sv->slot_req[k]->demand;
                in_step += 1;
            }
        const double limit = sv->admit_load * (double)sv->resident_warps;
        for (int k = 0; k < sv->max_slots && !sv->queue.empty(); ++k) {
            if (sv->slot_req[k]) continue;
            Request *r = sv->queue.front();
            if (r->cancelled) {
                sv->queue.pop_front();
                finish_locked(sv, r, ASYRK_ECANCELED);
                --k;
                continue;
            }
            if (in_step > 0 && sv->admit_load > 0.0 && (double)(demand + r->demand) > limit) break;
            if (!admit_locked(sv, r, k)) break;
            sv->queue.pop_front();
            demand += r->demand;
            in_step += 1;
        }
        int occupied = 0, oc = 0;
        for (int k = 0; k < sv->max_slots; ++k) occupied += sv->slot_req[k] ? 1 : 0;
        for (int k = 0; k < sv->oc_slots; ++k) oc += sv->oc_req[k] ? 1 : 0;
        if (occupied + oc > sv->max_active) sv->max_active = occupied + oc;
        if (occupied > sv->max_active_shared) sv->max_active_shared = occupied;
        if (sv->stop) {
            fail_shared_locked(sv, sv->fatal != ASYRK_OK ? sv->fatal : ASYRK_ECANCELED);
            break;
        }
        if (occupied == 0) {
            if (!sv->queue.empty())  // waits for memory the on-chip requests hold
                sv->cv_work.wait_for(lk, std::chrono::milliseconds(1), [&] { return sv->stop; });
            else
                sv->cv_work.wait_for(lk, std::chrono::milliseconds(50),
                                     [&] { return sv->stop || !sv->queue.empty(); });
            continue;
        }
        int st = engine_step(sv, lk, done);
        if (st == ASYRK_OK) st = harvest(sv, lk, done);
        if (st != ASYRK_OK) {
            sv->fatal = st;
            sv->stop = true;
            sv->cv_oc.notify_all();
            fail_shared_locked(sv, st);
            break;
        }
    }
}

// The on-chip requests' thread: FIFO admission into free on-chip slots while
// memory allows (each admission launches the request's solve on the slot's
// stream), and completion of the launches that have finished.
static void onchip_loop(asyrk_server *sv)
{
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        int next = 0;
        while (!sv->oc_queue.empty()) {
            Request *r = sv->oc_queue.front();
            if (r->cancelled) {
                sv->oc_queue.pop_front();
                finish_locked(sv, r, ASYRK_ECANCELED);
                continue;
            }
            while (next < sv->oc_slots && sv->oc_req[next]) ++next;
            if (next == sv->oc_slots || !admit_onchip_locked(sv, r, next)) break;
            sv->oc_queue.pop_front();
        }
        int in_flight = 0, shared = 0;
        for (int k = 0; k < sv->oc_slots; ++k) in_flight += sv->oc_req[k] ? 1 : 0;
        for (int k = 0; k < sv->max_slots; ++k) shared += sv->slot_req[k] ? 1 : 0;
        if (in_flight + shared > sv->max_active) sv->max_active = in_flight + shared;
        if (sv->stop || sv->fatal != ASYRK_OK) {
            const int why = sv->fatal != ASYRK_OK ? sv->fatal : ASYRK_ECANCELED;
            sv->stop = true;
            sv->cv_work.notify_all();
            fail_onchip_locked(sv, why);
            break;
        }
        if (in_flight == 0) {
            if (!sv->oc_queue.empty())  // waits for memory the shared step holds
                sv->cv_oc.wait_for(lk, std::chrono::milliseconds(1), [&] { return sv->stop; });
            else
                sv->cv_oc.wait_for(lk, std::chrono::milliseconds(50),
                                   [&] { return sv->stop || !sv->oc_queue.empty(); });
            continue;
        }
        bool any = false;
        const int st = harvest_onchip(sv, lk, &any);
        if (st != ASYRK_OK) {
            sv->fatal = st;
            continue;  // stops at the top of the loop
        }
        if (!any)  // launches in flight, none finished: look again shortly
            sv->cv_oc.wait_for(lk, std::chrono::microseconds(20), [&] { return sv->stop; });
    }
}

extern "C" int asyrk_server_create(asyrk_server **out, const asyrk_server_opts *opts)
{
    if (!out) return set_error(ASYRK_EINVAL, "out is NULL");
    *out = nullptr;
    asyrk_server_opts o;
    memset(&o, 0, sizeof o);
    if (opts) o = *opts;
    if (o.mem_budget_bytes <= 0) return set_error(ASYRK_EINVAL, "mem_budget_bytes must be > 0");
    if (o.max_slots < 0) return set_error(ASYRK_EINVAL, "max_slots < 0");
    if (o.row_exclusion < -1 || o.row_exclusion > 1)
        return set_error(ASYRK_EINVAL, "row_exclusion must be -1, 0 or 1");
    if (o.inner_tol < 0.0 || o.max_inner_sweeps < 0) return set_error(ASYRK_EINVAL, "bad inner solve limits");
    if (o.partition < -1) return set_error(ASYRK_EINVAL, "partition must be >= -1");
    if (!(o.admit_load == o.admit_load)) return set_error(ASYRK_EINVAL, "admit_load is NaN");
    asyrk_server *sv = new (std::nothrow) asyrk_server();
    if (!sv) return set_error(ASYRK_ENOMEM, "host allocation failed");
    auto fail = [&](int st) {
        if (sv->s && sv->s != sv->split.stream[0]) cudaStreamDestroy(sv->s);
        for (cudaStream_t x : sv->oc_stream) cudaStreamDestroy(x);
        sm_partition_destroy(&sv->split);
        for (cudaEvent_t x : sv->oc_ev) cudaEventDestroy(x);
        cudaFree(sv->oc_jobs);
        cudaFree(sv->d);
        delete sv->arena;
        delete sv;
        return st;
    };
    sv->budget = (size_t)o.mem_budget_bytes;
    sv->excl = o.row_exclusion >= 0;
    if (o.inner_tol > 0.0) sv->inner_tol = o.inner_tol;
    if (o.max_inner_sweeps > 0) sv->max_inner = o.max_inner_sweeps;
    if (o.admit_load != 0.0) sv->admit_load = o.admit_load > 0.0 ? o.admit_load : -1.0;
    cudaError_t e = cudaGetDevice(&sv->device);
    int sms = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, sv->device);
    if (e != cudaSuccess) return fail(cuda_fail(e, "device query", __FILE__, __LINE__));
    int st = batch_resident_warps(sms, sv->excl, &sv->resident_warps);
    if (st != ASYRK_OK) return fail(st);
    sv->max_slots = o.max_slots > 0 ? o.max_slots : 256;
    if (sv->max_slots > sv->resident_warps) sv->max_slots = sv->resident_warps;
    if (sv->max_slots > BATCH_MAX_SLOTS) sv->max_slots = BATCH_MAX_SLOTS;
    sv->onchip = o.onchip >= 0;
    sv->oc_slots = sv->onchip ? SERVER_ONCHIP_SLOTS : 0;
    sv->oc_req.assign(sv->oc_slots, nullptr);
    sv->oc_mem.assign(sv->oc_slots, SlotMem());
    sv->oc_hj.assign(sv->oc_slots, ClusterJob());
    sv->h.assign(sv->max_slots, SysDesc());
    memset(sv->h.data(), 0, sv->max_slots * sizeof(SysDesc));
    sv->slot_req.assign(sv->max_slots, nullptr);
    sv->slot_mem.assign(sv->max_slots, SlotMem());
    sv->arena = new (std::nothrow) Arena(sv->budget);
    if (!sv->arena) return fail(set_error(ASYRK_ENOMEM, "host allocation failed"));
    e = cudaMalloc((void **)&sv->d, sv->max_slots * sizeof(SysDesc));
    // on-chip requests on a few SMs of their own, the shared step on the rest:
    // the step's blocks then never wait for SMs the on-chip CTAs hold, and the
    // on-chip requests never wait for the step's blocks
    if (e == cudaSuccess && sv->oc_slots > 0 && o.partition >= 0) {
        const int oc_sms = o.partition > 0 ? o.partition : 16;
        if (oc_sms < sms && sm_partition_create(sv->device, sms - oc_sms, &sv->split)) {
            sv->s = sv->split.stream[0];
            sv->step_warps = (int)((long long)sv->resident_warps * sv->split.sms[0] / sms);
            if (sv->step_warps < 8) sv->step_warps = 8;
        }
    }
    if (e == cudaSuccess && !sv->s) e = cudaStreamCreateWithFlags(&sv->s, cudaStreamNonBlocking);
    if (e == cudaSuccess && sv->oc_slots > 0)
        e = cudaMalloc((void **)&sv->oc_jobs, sv->oc_slots * sizeof(ClusterJob));
    for (int k = 0; k < sv->oc_slots && e == cudaSuccess; ++k) {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        if (sv->split.ctx[1]) {
            if (!sm_partition_add_stream(sv->split, 1, &st)) e = cudaErrorUnknown;
        } else {
            e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        }
        if (e == cudaSuccess) sv->oc_stream.push_back(st);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) sv->oc_ev.push_back(ev);
    }
    if (e != cudaSuccess) return fail(cuda_fail(e, "server allocation", __FILE__, __LINE__));
    try {
        sv->th = std::thread(engine_loop, sv);
        if (sv->oc_slots > 0) sv->oc_th = std::thread(onchip_loop, sv);
    } catch (...) {
        if (sv->th.joinable()) {
            {
                std::lock_guard<std::mutex> lock(sv->mu);
                sv->stop = true;
                sv->cv_work.notify_all();
            }
            sv->th.join();
        }
        return fail(set_error(ASYRK_ENOMEM, "could not start the engine threads"));
    }
    *out = sv;
    return ASYRK_OK;
}

extern "C" int asyrk_server_submit(asyrk_server *sv, asyrk_problem *p, const double *x0,
                                   const double *x_true, double gamma, double tol, int mode,
                                   int64_t max_sweeps, uint64_t *ticket)
{
    if (!sv || !p || !ticket) return set_error(ASYRK_EINVAL, "NULL argument");
    if (p->dtype == ASYRK_F64)
        return set_error(ASYRK_EINVAL, "served solves take FP32 or BF16 values");
    if (mode != ASYRK_MODE_ASYNC && mode != ASYRK_MODE_REFINE)
        return set_error(ASYRK_EINVAL, "served mode must be ASYNC or REFINE");
    if (!(gamma > 0.0 && gamma < 2.0)) return set_error(ASYRK_EINVAL, "gamma must be in (0, 2)");
    if (!(tol > 0.0) || max_sweeps < 1) return set_error(ASYRK_EINVAL, "need tol > 0 and max_sweeps >= 1");
    Request *r = new (std::nothrow) Request();
    if (!r) return set_error(ASYRK_ENOMEM, "host allocation failed");
    r->p = p;
    r->x0.assign(p->n, 0.0);
    if (x0) memcpy(r->x0.data(), x0, p->n * sizeof(double));
    if (x_true) r->xt.assign(x_true, x_true + p->n);
    r->gamma = gamma;
    r->tol = tol;
    r->mode = mode;
    r->max_sweeps = max_sweeps;
    r->slot_bytes = request_bytes(p, x_true != nullptr, mode);
    memset(&r->info, 0, sizeof r->info);
    if (r->slot_bytes + (size_t)p->dev_bytes > sv->budget) {
        delete r;
        return set_error(ASYRK_ENOMEM, "the request needs %zu bytes, more than the whole budget",
                         (size_t)(request_bytes(p, x_true != nullptr, mode) + p->dev_bytes));
    }
    std::lock_guard<std::mutex> lock(sv->mu);
    if (sv->stop) {
        delete r;
        return sv->fatal != ASYRK_OK ? sv->fatal : set_error(ASYRK_EINVAL, "server is stopping");
    }
    // A problem that fits one CTA's shared memory, and whose Cor. 2 worker cap
    // a CTA's threads cover to within a factor 2 (one CTA would otherwise run
    // it slower than the shared step, whose projections take about twice as
    // long), is solved on-chip.
    if (sv->onchip) {
        ClusterShape sh;
        const int G = engine_subwarp(p, true);
        if (cluster_shape(p, G, 1, 0, &sh) == ASYRK_OK && sh.fits && sh.C == 1 &&
            tau_cap_estimate(p->m, p->n) <= 2LL * (CLUSTER_MAX_THREADS / G)) {
            const long long key = (long long)p->dtype * 64 + G;
            bool ok = true;
            if (std::find(sv->oc_prepared.begin(), sv->oc_prepared.end(), key) ==
                sv->oc_prepared.end()) {
                ok = cluster_prepare(p->dtype, G, 1) == ASYRK_OK;
                if (ok) sv->oc_prepared.push_back(key);
            }
            if (ok && cluster_check_schedulable(p->dtype, sh) == ASYRK_OK) {
                r->onchip = true;
                r->ocshape = sh;
            }
        }
    }
    if (!r->onchip) {
        const long long cw = (tau_cap_estimate(p->m, p->n) * engine_subwarp(p, false) + 31) / 32;
        r->demand = cw < 1 ? 1 : cw > sv->resident_warps ? sv->resident_warps : cw;
    }
    r->ticket = sv->next_ticket++;
    r->t_submit = now_s();
    (r->onchip ? sv->oc_queue : sv->queue).push_back(r);
    sv->reqs[r->ticket] = r;
    sv->submitted += 1;
    *ticket = r->ticket;
    (r->onchip ? sv->cv_oc : sv->cv_work).notify_one();
    return ASYRK_OK;
}

extern "C" int asyrk_server_wait(asyrk_server *sv, uint64_t ticket, double *x,
                                 asyrk_solve_info *info, int64_t timeout_us)
{
    if (!sv) return set_error(ASYRK_EINVAL, "NULL server");
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return set_error(ASYRK_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
    Request *r = it->second;
    if (timeout_us < 0) {
        sv->cv_done.wait(lk, [&] { return r->done; });
    } else if (!sv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return r->done; })) {
        return set_error(ASYRK_ETIMEOUT, "request %llu not finished", (unsigned long long)ticket);
    }
    if (x && !r->result.empty()) memcpy(x, r->result.data(), r->result.size() * sizeof(double));
    if (info) *info = r->info;
    const int st = r->status;
    sv->reqs.erase(it);
    delete r;
    return st;
}

extern "C" int asyrk_server_cancel(asyrk_server *sv, uint64_t ticket)
{
    if (!sv) return set_error(ASYRK_EINVAL, "NULL server");
    std::lock_guard<std::mutex> lock(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return set_error(ASYRK_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
    Request *r = it->second;
    if (r->done) return ASYRK_OK;
    r->cancelled = true;
    std::deque<Request *> &q = r->onchip ? sv->oc_queue : sv->queue;
    for (auto it = q.begin(); it != q.end(); ++it) {
        if (*it == r) {
            q.erase(it);
            finish_locked(sv, r, ASYRK_ECANCELED);
            break;
        }
    }
    (r->onchip ? sv->cv_oc : sv->cv_work).notify_one();
    return ASYRK_OK;
}

extern "C" int asyrk_server_get_stats(asyrk_server *sv, asyrk_server_stats *st)
{
    if (!sv || !st) return set_error(ASYRK_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(sv->mu);
    memset(st, 0, sizeof *st);
    st->submitted = sv->submitted;
    st->completed = sv->completed;
    st->queued = (int64_t)(sv->queue.size() + sv->oc_queue.size());
    int64_t act = 0;
    for (auto *r : sv->slot_req) act += r ? 1 : 0;
    for (auto *r : sv->oc_req) act += r ? 1 : 0;
    st->active = act;
    st->onchip_completed = sv->oc_completed;
    st->iterations = sv->iterations;
    st->kernel_launches = sv->launches;
    st->mem_used = (int64_t)sv->used;
    st->mem_budget = (int64_t)sv->budget;
    st->arena_reserved = (int64_t)sv->arena->reserved();
    st->max_slots = sv->max_slots;
    st->max_active = (int32_t)sv->max_active;
    st->max_active_shared = (int32_t)sv->max_active_shared;
    st->step_sms = sv->split.sms[0];
    st->onchip_sms = sv->split.sms[1];
    st->fatal = sv->fatal;
    return ASYRK_OK;
}

extern "C" void asyrk_server_destroy(asyrk_server *sv)
{
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        sv->stop = true;
        sv->cv_work.notify_all();
        sv->cv_oc.notify_all();
    }
    if (sv->th.joinable()) sv->th.join();
    if (sv->oc_th.joinable()) sv->oc_th.join();
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        fail_shared_locked(sv, ASYRK_ECANCELED);
        fail_onchip_locked(sv, ASYRK_ECANCELED);
        for (auto &kv : sv->reqs) delete kv.second;
        sv->reqs.clear();
    }
    cudaStreamSynchronize(sv->s);
    if (sv->s != sv->split.stream[0]) cudaStreamDestroy(sv->s);
    for (cudaStream_t x : sv->oc_stream) cudaStreamDestroy(x);
    sm_partition_destroy(&sv->split);
    for (cudaEvent_t x : sv->oc_ev) cudaEventDestroy(x);
    cudaFree(sv->oc_jobs);
    cudaFree(sv->d);
    cudaFree(sv->part);
    delete sv->arena;
    delete sv;
}
