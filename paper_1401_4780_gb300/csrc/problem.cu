// problem.cu -- asyrk_create / asyrk_destroy and the problem set-up on the GPU.
//
// Set-up of a problem (Section 1 of the paper: A x = b consistent, no zero
// rows; rows are drawn with probability ||a_i||^2/||A||_F^2):
//   1. a GPU pass over row_ptr checks it (rp[0] = 0, no empty row, no row
//      longer than n) and a prefix sum gives the padded row starts (rows
//      rounded up to 4 entries);
//   2. a GPU pass over the rows checks columns (strictly ascending, in range)
//      and values (finite), computes w_i = ||a_i||^2 in FP64 in CSR order
//      without fused multiply-adds, and writes the row records and the
//      padded column/value arrays;
//   3. ||A||_F^2, ||b|| and the alias table of the w_i (as specified in
//      asyrk.h) are computed on the GPU (alias.cu) and written into the
//      records.  The host only reads back sizes, flags and the totals.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>


#include "alias.cuh"
#include "common.cuh"
#include "devmem.cuh"
#include "scan.cuh"

namespace asyrk {

static thread_local char g_last_error[512] = "";

int set_error(int status, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof g_last_error, fmt, ap);
    va_end(ap);
    return status;
}

int cuda_fail(cudaError_t e, const char *what, const char *file, int line)
{
    const char *base = strrchr(file, '/');
    int st = (e == cudaErrorMemoryAllocation) ? ASYRK_ENOMEM : ASYRK_ECUDA;
    return set_error(st, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e),
                     base ? base + 1 : file, line);
}

template <typename T>
static int dev_alloc(asyrk_problem *p, T **ptr, size_t count, cudaStream_t s)
{
    if (count == 0) count = 1;
    const int st = devmem_alloc_n(ptr, count, s);
    if (st != ASYRK_OK) return st;
    p->dev_bytes += (int64_t)(count * sizeof(T));
    return ASYRK_OK;
}

// error bits raised by the row pass
enum : unsigned {
    ERR_COL_RANGE = 1u,
    ERR_COL_ORDER = 2u,
    ERR_VAL = 4u,
    ERR_ZERO_ROW = 8u,
    ERR_B = 16u,
};

__device__ __forceinline__ double widen(double v) { return v; }
__device__ __forceinline__ double widen(float v) { return (double)v; }
__device__ __forceinline__ double widen(bf16_t v)
{
    return (double)__uint_as_float(((unsigned)v.bits) << 16);
}

template <typename VT>
__device__ __forceinline__ bool finite_val(VT v)
{
    return isfinite(widen(v));
}

// One thread per row.  src_* index the caller's CSR layout, dst_* the padded
// one; when no padding is needed src and dst are the same arrays.
template <typename VT>
__global__ void k_row_setup(int64_t r0, int64_t r1, int64_t n, const int64_t *__restrict__ row_ptr,
                            const int64_t *__restrict__ pstart, const int32_t *src_col,
                            const VT *src_val, int32_t *dst_col, VT *dst_val,
                            const double *__restrict__ b, RowRec *__restrict__ rec,
                            double *__restrict__ w64, double *__restrict__ b64,
                            unsigned *__restrict__ err)
{
    const int64_t i = r0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // rows [r0, r1)
    if (i >= r1) return;
    const int64_t s = row_ptr[i], e = row_ptr[i + 1];
    const int64_t d = pstart ? pstart[i] : s;
    unsigned bad = 0;
    double w = 0.0;
    int32_t prev = -1;
    for (int64_t k = s; k < e; ++k) {
        const int32_t c = src_col[k];
        const VT v = src_val[k];
        if (c < 0 || (int64_t)c >= n) bad |= ERR_COL_RANGE;
        if (c <= prev) bad |= ERR_COL_ORDER;
        prev = c;
        if (!finite_val(v)) bad |= ERR_VAL;
        const double dv = widen(v);
        w = __dadd_rn(w, __dmul_rn(dv, dv));
        if (pstart) {
            dst_col[d + (k - s)] = c;
            dst_val[d + (k - s)] = v;
        }
    }
    const int64_t len = e - s;
    if (pstart) {  // zero the padding up to the next multiple of 4
        const int64_t padded = (len + 3) & ~(int64_t)3;
        for (int64_t k = len; k < padded; ++k) {
            dst_col[d + k] = 0;
            VT z;
            memset(&z, 0, sizeof z);
            dst_val[d + k] = z;
        }
    }
    if (!(w > 0.0) || !isfinite(w)) bad |= ERR_ZERO_ROW;
    const double bi = b[i];
    if (!isfinite(bi)) bad |= ERR_B;
    if (bad) atomicOr(err, bad);
    RowRec r;
    r.start = d;
    r.len = (unsigned)len;
    r.thr = 0xffffffffu;
    r.alias = (unsigned)i;
    r.b = (float)bi;
    r.inv = (float)(1.0 / w);
    r.pad = 0u;
    rec[i] = r;
    w64[i] = w;
    b64[i] = bi;
}


static size_t value_size(int dtype)
{
    return dtype == ASYRK_F64 ? 8 : dtype == ASYRK_F32 ? 4 : 2;
}

template <typename VT>
static void launch_row_setup(asyrk_problem *p, int64_t r0, int64_t r1, const int64_t *row_ptr_d,
                             const int64_t *pstart_d, const int32_t *src_col, const void *src_val,
                             const double *b_d, unsigned *err_d, cudaStream_t s)
{
    const int T = 256;
    const int64_t blocks = (r1 - r0 + T - 1) / T;
    k_row_setup<VT><<<(unsigned)blocks, T, 0, s>>>(
        r0, r1, p->n, row_ptr_d, pstart_d, src_col, (const VT *)src_val, p->col, (VT *)p->val, b_d,
        p->rec, p->w64, p->b64, err_d);
}

static void row_setup(asyrk_problem *p, int64_t r0, int64_t r1, const int64_t *row_ptr_d,
                      const int64_t *pstart_d, const int32_t *src_col, const void *src_val,
                      const double *b_d, unsigned *err_d, cudaStream_t s)
{
    if (r1 <= r0) return;
    switch (p->dtype) {
    case ASYRK_F64: launch_row_setup<double>(p, r0, r1, row_ptr_d, pstart_d, src_col, src_val, b_d, err_d, s); break;
    case ASYRK_F32: launch_row_setup<float>(p, r0, r1, row_ptr_d, pstart_d, src_col, src_val, b_d, err_d, s); break;
    default: launch_row_setup<bf16_t>(p, r0, r1, row_ptr_d, pstart_d, src_col, src_val, b_d, err_d, s); break;
    }
}

// Host entries go to the device in chunks of about CREATE_CHUNK_BYTES on a
// stream of their own, while the row pointers are checked and the rows of each
// chunk that has arrived are set up.
constexpr int64_t CREATE_CHUNK_BYTES = 64LL << 20;
constexpr int CREATE_MAX_CHUNKS = 32;
// entries a problem may have: every byte count below stays inside int64
constexpr int64_t CREATE_MAX_NNZ = 1LL << 58;

// first entry of chunk c of `chunks` over nnz entries
static int64_t chunk_begin(int64_t nnz, int chunks, int c)
{
    const int64_t q = nnz / chunks, r = nnz % chunks;
    return q * c + (c < r ? c : r);
}

int ensure_workspace(asyrk_problem *p)
{
    if (p->ev[1]) return ASYRK_OK;
    int st;
    const size_t words = (size_t)((p->m + 31) / 32);
    if (!p->xw && (st = dev_alloc(p, (double **)&p->xw, (size_t)p->n, nullptr)) != ASYRK_OK) return st;
    if (!p->x64 && (st = dev_alloc(p, &p->x64, (size_t)p->n, nullptr)) != ASYRK_OK) return st;
    if (!p->xt64 && (st = dev_alloc(p, &p->xt64, (size_t)p->n, nullptr)) != ASYRK_OK) return st;
    if (!p->red_part &&
        (st = dev_alloc(p, &p->red_part, (size_t)ASYRK_MAX_RED_BLOCKS * 4, nullptr)) != ASYRK_OK)
        return st;
    if (!p->red_count) {
        if ((st = dev_alloc(p, &p->red_count, 1, nullptr)) != ASYRK_OK) return st;
        ASYRK_CK(cudaMemset(p->red_count, 0, sizeof(unsigned)));
    }
    if (!p->red_out && (st = dev_alloc(p, &p->red_out, 8, nullptr)) != ASYRK_OK) return st;
    if (!p->busy) {
        if ((st = dev_alloc(p, &p->busy, words, nullptr)) != ASYRK_OK) return st;
        ASYRK_CK(cudaMemset(p->busy, 0, words * sizeof(unsigned)));
    }
    if (!p->skipped && (st = dev_alloc(p, &p->skipped, 1, nullptr)) != ASYRK_OK) return st;
    ASYRK_CK(cudaStreamSynchronize(nullptr));  // the allocations, ordered on that stream
    if (!p->h_out) ASYRK_CK(cudaMallocHost((void **)&p->h_out, 8 * sizeof(double)));
    if (!p->ev[0]) ASYRK_CK(cudaEventCreate(&p->ev[0]));
    if (!p->ev[1]) ASYRK_CK(cudaEventCreate(&p->ev[1]));
    return ASYRK_OK;
}

static void free_problem(asyrk_problem *p)
{
    if (!p) return;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != p->device) cudaSetDevice(p->device);
    // no work that uses the handle's memory may still run (cudaFree used to
    // wait for the device the same way); the memory goes back to the pool
    cudaDeviceSynchronize();
    void *mem[] = {p->rec, p->col, p->val, p->b64, p->w64, p->xw, p->x64, p->xt64, p->g64,
                   p->red_part, p->red_count, p->red_out, p->rows_buf, p->busy, p->skipped,
                   p->loop_state};
    for (void *q : mem) devmem_free(q, nullptr);
    if (p->h_out) cudaFreeHost(p->h_out);
    if (p->ev[0]) cudaEventDestroy(p->ev[0]);
    if (p->ev[1]) cudaEventDestroy(p->ev[1]);
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    if (cur >= 0 && cur != p->device) cudaSetDevice(cur);
    delete p;
}

// Row-pointer pass: rp[0] = 0, every row non-empty and at most n long; the
// padded length of each row (a multiple of 4 entries) and the row lengths'
// maximum; whether every row already starts at a multiple of 4.
enum : unsigned { RP_FIRST = 1u, RP_EMPTY = 2u, RP_LONG = 4u, RP_MISALIGNED = 8u };

constexpr int RP_THREADS = 256;

__global__ void __launch_bounds__(RP_THREADS) k_rowptr_pass(int64_t m, int64_t n,
                                                           const int64_t *__restrict__ rp,
                                                           int64_t *__restrict__ plen,
                                                           unsigned long long *__restrict__ info)
{
    // info[0]: flags, info[1]: max row length, info[2]: first bad row.  Flags and
    // the maximum are reduced over the block first: one atomic per block rather
    // than one per row on a single address.
    __shared__ unsigned s_len[RP_THREADS / 32], s_flag[RP_THREADS / 32];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned f = 0, l32 = 0;
    if (i < m) {
        const int64_t s = rp[i], len = rp[i + 1] - s;
        if (i == 0 && s != 0) f |= RP_FIRST;
        if (len <= 0) f |= RP_EMPTY;
        if (len > n) f |= RP_LONG;
        if (s & 3) f |= RP_MISALIGNED;
        plen[i] = len > 0 ? ((len + 3) & ~(int64_t)3) : 0;
        l32 = len <= 0 ? 0u : len > 0xffffffffLL ? 0xffffffffu : (unsigned)len;
        if (f & (RP_FIRST | RP_EMPTY | RP_LONG)) atomicMin(&info[2], (unsigned long long)i);
    }
    l32 = __reduce_max_sync(0xffffffffu, l32);
    f = __reduce_or_sync(0xffffffffu, f);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { s_len[w] = l32; s_flag[w] = f; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < RP_THREADS / 32; ++k) {
            l32 = max(l32, s_len[k]);
            f |= s_flag[k];
        }
        if (l32) atomicMax(&info[1], (unsigned long long)l32);
        if (f) atomicOr(&info[0], (unsigned long long)f);
    }
}

static int create_impl(asyrk_problem *p, const int64_t *row_ptr, const int32_t *col_idx,
                       const void *values, const double *b, const asyrk_create_opts *o)
{
    const int64_t m = p->m, n = p->n;
    const bool on_dev = o->device_ptrs != 0;
    cudaStream_t s = (cudaStream_t)o->stream;
    ASYRK_CK(cudaGetDevice(&p->device));
    ASYRK_CK(cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device));

    // temporaries, freed on every exit path
    int64_t *rp_d = nullptr, *ps_d = nullptr, *plen_d = nullptr, *scan_tmp = nullptr;
    unsigned long long *info_d = nullptr;
    int32_t *col_src = nullptr;
    void *val_src = nullptr;
    double *b_d = nullptr;
    unsigned *err_d = nullptr;
    bool own_src = false;
    cudaStream_t cs = nullptr;  // the host entries' copies
    cudaEvent_t ev_go = nullptr, ev_chunk[CREATE_MAX_CHUNKS] = {};
    int chunks = 0;
    auto cleanup = [&]() {
        // copies still in flight end before their buffers go back to the pool,
        // which takes them in the order of the stream that used them
        if (cs) cudaStreamSynchronize(cs);
        if (!on_dev) { devmem_free(rp_d, s); devmem_free(b_d, s); }
        if (own_src) { devmem_free(col_src, s); devmem_free(val_src, s); }
        devmem_free(ps_d, s); devmem_free(plen_d, s); devmem_free(scan_tmp, s);
        devmem_free(info_d, s); devmem_free(err_d, s);
        for (cudaEvent_t e : ev_chunk)
            if (e) cudaEventDestroy(e);
        if (ev_go) cudaEventDestroy(ev_go);
        if (cs) cudaStreamDestroy(cs);
    };
    auto fail = [&](int code) { cleanup(); return code; };
#define ASYRK_ALLOC(ptr, bytes)                                                            \
    do {                                                                                   \
        const int st__ = devmem_alloc((void **)&(ptr), (bytes), s);                        \
        if (st__ != ASYRK_OK) return fail(st__);                                           \
    } while (0)
#define ASYRK_CKC(call)                                                                    \
    do {                                                                                   \
        cudaError_t e__ = (call);                                                          \
        if (e__ != cudaSuccess) return fail(cuda_fail(e__, #call, __FILE__, __LINE__));    \
    } while (0)

    // 1. row pointers on the device (checked below)
    if (on_dev) {
        rp_d = const_cast<int64_t *>(row_ptr);
    } else {
        ASYRK_ALLOC(rp_d, (m + 1) * sizeof(int64_t));
        ASYRK_CKC(cudaMemcpyAsync(rp_d, row_ptr, (m + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    }

    // 2. host entries and b on their way while the row pointers are checked.
    //    The arrays hold row_ptr[m] entries (the caller's contract; the device
    //    copy's row_ptr[m] is compared below); chunk c is a contiguous range of
    //    entries, copied on cs after the row pointers.
    const size_t es = value_size(p->dtype);
    int64_t nnz_h = 0;
    if (!on_dev) {
        if (row_ptr[0] != 0) return fail(set_error(ASYRK_EINVAL, "row_ptr[0] must be 0"));
        nnz_h = row_ptr[m];
        if (nnz_h < m || nnz_h > m * n || nnz_h > CREATE_MAX_NNZ)
            return fail(set_error(ASYRK_EINVAL, "row_ptr[m] = %lld: every row needs an entry and "
                                  "at most n", (long long)nnz_h));
        own_src = true;
        ASYRK_ALLOC(col_src, (size_t)nnz_h * 4);
        ASYRK_ALLOC(val_src, (size_t)nnz_h * es);
        ASYRK_ALLOC(b_d, m * sizeof(double));
        ASYRK_CKC(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        ASYRK_CKC(cudaEventCreateWithFlags(&ev_go, cudaEventDisableTiming));
        ASYRK_CKC(cudaEventRecord(ev_go, s));  // the allocations, the row pointers' copy
        ASYRK_CKC(cudaStreamWaitEvent(cs, ev_go, 0));
        ASYRK_CKC(cudaMemcpyAsync(b_d, b, m * sizeof(double), cudaMemcpyHostToDevice, cs));
        const int64_t bytes = nnz_h * (int64_t)(4 + es);
        chunks = (int)std::min<int64_t>(CREATE_MAX_CHUNKS,
                                        std::max<int64_t>(1, (bytes + CREATE_CHUNK_BYTES - 1) /
                                                                 CREATE_CHUNK_BYTES));
        for (int c = 0; c < chunks; ++c) {
            const int64_t z0 = chunk_begin(nnz_h, chunks, c), z1 = chunk_begin(nnz_h, chunks, c + 1);
            ASYRK_CKC(cudaMemcpyAsync(col_src + z0, col_idx + z0, (size_t)(z1 - z0) * 4,
                                      cudaMemcpyHostToDevice, cs));
            ASYRK_CKC(cudaMemcpyAsync((char *)val_src + (size_t)z0 * es,
                                      (const char *)values + (size_t)z0 * es, (size_t)(z1 - z0) * es,
                                      cudaMemcpyHostToDevice, cs));
            ASYRK_CKC(cudaEventCreateWithFlags(&ev_chunk[c], cudaEventDisableTiming));
            ASYRK_CKC(cudaEventRecord(ev_chunk[c], cs));
        }
    }

    // 3. row-pointer checks, padded row starts (a prefix sum)
    ASYRK_ALLOC(plen_d, m * sizeof(int64_t));
    ASYRK_ALLOC(ps_d, (m + 1) * sizeof(int64_t));
    ASYRK_ALLOC(scan_tmp, scan_tmp_count(m) * sizeof(int64_t));
    ASYRK_ALLOC(info_d, 3 * sizeof(unsigned long long));
    ASYRK_CKC(cudaMemsetAsync(info_d, 0, 2 * sizeof(unsigned long long), s));
    ASYRK_CKC(cudaMemsetAsync(info_d + 2, 0xff, sizeof(unsigned long long), s));
    k_rowptr_pass<<<(unsigned)((m + RP_THREADS - 1) / RP_THREADS), RP_THREADS, 0, s>>>(m, n, rp_d, plen_d, info_d);
    ASYRK_CKC(cudaGetLastError());
    int st = exclusive_scan(plen_d, ps_d, m, scan_tmp, ps_d + m, s);
    if (st != ASYRK_OK) return fail(st);
    unsigned long long info[3];
    int64_t tail[2];  // rp[m], padded total
    ASYRK_CKC(cudaMemcpyAsync(info, info_d, sizeof info, cudaMemcpyDeviceToHost, s));
    ASYRK_CKC(cudaMemcpyAsync(&tail[0], rp_d + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    ASYRK_CKC(cudaMemcpyAsync(&tail[1], ps_d + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    ASYRK_CKC(cudaStreamSynchronize(s));
    if (info[0] & RP_FIRST) return fail(set_error(ASYRK_EINVAL, "row_ptr[0] must be 0"));
    if (info[0] & RP_EMPTY)
        return fail(set_error(ASYRK_EINVAL, "row %llu is empty or row_ptr decreases (the problem "
                              "has no zero rows)", info[2]));
    if (info[0] & RP_LONG) return fail(set_error(ASYRK_EINVAL, "a row has more entries than n"));
    if (!on_dev && tail[0] != nnz_h)
        return fail(set_error(ASYRK_EINVAL, "row_ptr changed while the problem was created"));
    if (tail[1] > CREATE_MAX_NNZ) return fail(set_error(ASYRK_ENOMEM, "too many entries"));
    const bool aligned = !(info[0] & RP_MISALIGNED) && tail[1] == tail[0];
    p->nnz = tail[0];
    p->nnz_pad = aligned ? p->nnz : tail[1];
    p->max_len = (int64_t)info[1];

    // 4. device arrays; staged host entries whose rows are already 4-aligned
    //    are the handle's arrays as they stand
    if (aligned && own_src) {
        p->col = col_src;
        p->val = val_src;
        own_src = false;
    } else {
        if ((st = dev_alloc(p, &p->col, (size_t)p->nnz_pad, s)) != ASYRK_OK) return fail(st);
        if ((st = dev_alloc(p, (char **)&p->val, (size_t)p->nnz_pad * es, s)) != ASYRK_OK) return fail(st);
    }
    if ((st = dev_alloc(p, &p->rec, (size_t)m, s)) != ASYRK_OK) return fail(st);
    if ((st = dev_alloc(p, &p->b64, (size_t)m, s)) != ASYRK_OK) return fail(st);
    if ((st = dev_alloc(p, &p->w64, (size_t)m, s)) != ASYRK_OK) return fail(st);
    ASYRK_ALLOC(err_d, sizeof(unsigned));
    ASYRK_CKC(cudaMemsetAsync(err_d, 0, sizeof(unsigned), s));

    // 5. the row pass: checks, row weights and records, and the padding copy
    //    when rows are not 4-aligned; on host entries, the rows of each chunk
    //    once it has arrived (rows that reach into chunk c wait for it)
    const int64_t *pstart = aligned ? nullptr : ps_d;
    if (on_dev) {
        const int32_t *rs_col = col_idx;
        const void *rs_val = values;
        if (aligned) {
            ASYRK_CKC(cudaMemcpyAsync(p->col, col_idx, p->nnz * 4, cudaMemcpyDeviceToDevice, s));
            ASYRK_CKC(cudaMemcpyAsync(p->val, values, p->nnz * es, cudaMemcpyDeviceToDevice, s));
            rs_col = p->col;
            rs_val = p->val;
        }
        row_setup(p, 0, m, rp_d, pstart, rs_col, rs_val, b, err_d, s);
    } else {
        const int32_t *rs_col = aligned ? p->col : col_src;
        const void *rs_val = aligned ? p->val : val_src;
        int64_t r0 = 0;
        for (int c = 0; c < chunks; ++c) {
            // rows whose entries lie in chunks 0..c: row_ptr[i+1] <= the chunk's end
            const int64_t z1 = chunk_begin(p->nnz, chunks, c + 1);
            const int64_t r1 = c == chunks - 1
                                   ? m
                                   : (int64_t)(std::upper_bound(row_ptr + 1, row_ptr + m + 1, z1) -
                                               (row_ptr + 1));
            ASYRK_CKC(cudaStreamWaitEvent(s, ev_chunk[c], 0));
            row_setup(p, r0, r1, rp_d, pstart, rs_col, rs_val, b_d, err_d, s);
            r0 = r1;
        }
    }
    ASYRK_CKC(cudaGetLastError());
    unsigned err_h = 0;
    ASYRK_CKC(cudaMemcpyAsync(&err_h, err_d, sizeof err_h, cudaMemcpyDeviceToHost, s));
    ASYRK_CKC(cudaStreamSynchronize(s));
    if (err_h) {
        const char *why = (err_h & ERR_COL_RANGE)  ? "a column index is outside [0, n)"
                          : (err_h & ERR_COL_ORDER) ? "columns are not strictly ascending within a row"
                          : (err_h & ERR_VAL)       ? "a value is not finite"
                          : (err_h & ERR_ZERO_ROW)  ? "a row has zero norm (the problem has no zero rows)"
                                                    : "b has a non-finite entry";
        return fail(set_error(ASYRK_EINVAL, "malformed problem: %s", why));
    }

    // 6. ||A||_F^2, ||b|| and the alias table of the row weights, on the GPU
    if ((st = row_totals_and_alias(p, s)) != ASYRK_OK) return fail(st);
    cleanup();
#undef ASYRK_CKC
#undef ASYRK_ALLOC
    return ASYRK_OK;
}

}  // namespace asyrk

using namespace asyrk;

extern "C" int asyrk_create(asyrk_problem **out, int64_t m, int64_t n, const int64_t *row_ptr,
                            const int32_t *col_idx, const void *values, int vdtype,
                            const double *b, const asyrk_create_opts *opts)
{
    if (!out) return set_error(ASYRK_EINVAL, "out is NULL");
    *out = nullptr;
    if (m <= 0 || n <= 0 || m > 0x7fffffffLL || n > 0x7fffffffLL)
        return set_error(ASYRK_EINVAL, "m and n must be in [1, 2^31-1]");
    if (!row_ptr || !col_idx || !values || !b) return set_error(ASYRK_EINVAL, "NULL array");
    if (vdtype != ASYRK_F64 && vdtype != ASYRK_F32 && vdtype != ASYRK_BF16)
        return set_error(ASYRK_EINVAL, "unknown value dtype %d", vdtype);
    asyrk_create_opts o;
    memset(&o, 0, sizeof o);
    if (opts) o = *opts;
    if (o.reserved != 0) return set_error(ASYRK_EINVAL, "reserved option field must be 0");
    asyrk_problem *p = new (std::nothrow) asyrk_problem();
    if (!p) return set_error(ASYRK_ENOMEM, "host allocation failed");
    p->m = m;
    p->n = n;
    p->dtype = vdtype;
    p->seed = o.seed;
    int st = create_impl(p, row_ptr, col_idx, values, b, &o);
    if (st != ASYRK_OK) {
        free_problem(p);
        return st;
    }
    *out = p;
    return ASYRK_OK;
}

extern "C" void asyrk_destroy(asyrk_problem *p) { free_problem(p); }

extern "C" int asyrk_get_position(asyrk_problem *p, uint64_t *j_next)
{
    if (!p || !j_next) return set_error(ASYRK_EINVAL, "NULL argument");
    *j_next = p->j_next;
    return ASYRK_OK;
}

extern "C" int asyrk_set_position(asyrk_problem *p, uint64_t j_next)
{
    if (!p) return set_error(ASYRK_EINVAL, "NULL problem");
    p->j_next = j_next;
    return ASYRK_OK;
}

extern "C" int asyrk_problem_get_stats(asyrk_problem *p, asyrk_problem_stats *st)
{
    if (!p || !st) return set_error(ASYRK_EINVAL, "NULL argument");
    memset(st, 0, sizeof *st);
    st->m = p->m;
    st->n = p->n;
    st->nnz = p->nnz;
    st->nnz_padded = p->nnz_pad;
    st->max_row_len = p->max_len;
    st->device_bytes = p->dev_bytes;
    st->frob2 = p->frob2;
    st->dtype = p->dtype;
    st->uniform = p->uniform;
    st->seed = p->seed;
    st->j_next = p->j_next;
    return ASYRK_OK;
}

extern "C" int asyrk_draw_rows(asyrk_problem *p, uint64_t j0, int64_t count, uint32_t stream_id,
                               int sampling, int32_t *rows_out)
{
    if (!p || (count > 0 && !rows_out) || count < 0 || sampling < 0 || sampling > 1)
        return set_error(ASYRK_EINVAL, "bad argument");
    if (count == 0) return ASYRK_OK;
    if (count > p->rows_cap) {
        // the legacy default stream orders these with the launch and copy below
        devmem_free(p->rows_buf, nullptr);
        p->rows_buf = nullptr;
        p->rows_cap = 0;
        const int st = devmem_alloc_n(&p->rows_buf, (size_t)count, nullptr);
        if (st != ASYRK_OK) return st;
        p->rows_cap = count;
    }
    int st = launch_draw_rows(p, j0, count, stream_id, sampling, p->rows_buf, 0);
    if (st != ASYRK_OK) return st;
    ASYRK_CK(cudaMemcpy(rows_out, p->rows_buf, count * sizeof(int32_t), cudaMemcpyDeviceToHost));
    return ASYRK_OK;
}

extern "C" const char *asyrk_strerror(int status)
{
    switch (status) {
    case ASYRK_OK: return "ok";
    case ASYRK_EINVAL: return "invalid argument or malformed problem";
    case ASYRK_ENOMEM: return "out of memory";
    case ASYRK_ECUDA: return "CUDA error";
    case ASYRK_ETIMEOUT: return "timed out";
    case ASYRK_ECANCELED: return "cancelled";
    case ASYRK_NOT_CONVERGED: return "tolerance not reached within max_sweeps";
    case ASYRK_DIVERGED: return "iteration diverged";
    default: return "unknown status";
    }
}

extern "C" const char *asyrk_last_error(void) { return asyrk::g_last_error; }

extern "C" int asyrk_abi_version(void) { return ASYRK_ABI_VERSION; }
