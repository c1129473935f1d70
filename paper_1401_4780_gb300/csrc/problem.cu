// problem.cu -- asyrk_create / asyrk_destroy and the problem set-up on the GPU.
//
// Set-up of a problem (Section 1 of the paper: A x = b consistent, no zero
// rows; rows are drawn with probability ||a_i||^2/||A||_F^2):
//   1. row_ptr is checked on the host and the padded row starts (rounded up
//      to 4 entries) are computed;
//   2. a GPU pass over the rows checks columns (strictly ascending, in range)
//      and values (finite), computes w_i = ||a_i||^2 in FP64 in CSR order
//      without fused multiply-adds, and writes the row records and the
//      padded column/value arrays;
//   3. the host builds Vose's alias table of the w_i (the same specification
//      as documented in asyrk.h) and the GPU merges it into the records.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "common.cuh"

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
static int dev_alloc(asyrk_problem *p, T **ptr, size_t count)
{
    *ptr = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)ptr, count * sizeof(T));
    if (e != cudaSuccess) {
        *ptr = nullptr;
        (void)cudaGetLastError();
        return set_error(ASYRK_ENOMEM, "cudaMalloc of %zu bytes failed: %s",
                         count * sizeof(T), cudaGetErrorString(e));
    }
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
__global__ void k_row_setup(int64_t m, int64_t n, const int64_t *__restrict__ row_ptr,
                            const int64_t *__restrict__ pstart, const int32_t *src_col,
                            const VT *src_val, int32_t *dst_col, VT *dst_val,
                            const double *__restrict__ b, RowRec *__restrict__ rec,
                            double *__restrict__ w64, double *__restrict__ b64,
                            unsigned *__restrict__ err)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
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

__global__ void k_set_alias(int64_t m, const uint2 *__restrict__ tab, RowRec *__restrict__ rec)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const uint2 t = tab[i];
    rec[i].thr = t.x;
    rec[i].alias = t.y;
}

// Vose's method, in the order stated in asyrk.h: q_i = w_i m / F; "small"
// (q < 1) and "large" (q >= 1) stacks filled in ascending i; pair the top of
// small with the top of large; the large entry's q absorbs the deficit and
// moves to small once below 1; leftovers keep thr = 2^32-1 and themselves.
// Returns true when all weights are bit-identical (no table needed).
static bool build_alias(const std::vector<double> &w, double F, std::vector<uint2> &tab)
{
    const size_t m = w.size();
    tab.resize(m);
    for (size_t i = 0; i < m; ++i) tab[i] = make_uint2(0xffffffffu, (unsigned)i);
    bool same = true;
    for (size_t i = 1; i < m && same; ++i) same = (memcmp(&w[i], &w[0], sizeof(double)) == 0);
    if (same) return true;
    std::vector<double> q(m);
    std::vector<size_t> small, large;
    small.reserve(m);
    large.reserve(m);
    const double md = (double)m;
    for (size_t i = 0; i < m; ++i) {
        q[i] = (w[i] * md) / F;
        (q[i] < 1.0 ? small : large).push_back(i);
    }
    while (!small.empty() && !large.empty()) {
        const size_t s = small.back();
        small.pop_back();
        const size_t l = large.back();
        const double scaled = floor(q[s] * 4294967296.0);
        tab[s].x = scaled >= 4294967295.0 ? 0xffffffffu : (unsigned)scaled;
        tab[s].y = (unsigned)l;
        q[l] = (q[l] + q[s]) - 1.0;
        if (q[l] < 1.0) {
            large.pop_back();
            small.push_back(l);
        }
    }
    return false;
}

static size_t value_size(int dtype)
{
    return dtype == ASYRK_F64 ? 8 : dtype == ASYRK_F32 ? 4 : 2;
}

template <typename VT>
static void launch_row_setup(asyrk_problem *p, const int64_t *row_ptr_d, const int64_t *pstart_d,
                             const int32_t *src_col, const void *src_val, const double *b_d,
                             unsigned *err_d, cudaStream_t s)
{
    const int T = 256;
    const int64_t blocks = (p->m + T - 1) / T;
    k_row_setup<VT><<<(unsigned)blocks, T, 0, s>>>(
        p->m, p->n, row_ptr_d, pstart_d, src_col, (const VT *)src_val, p->col, (VT *)p->val, b_d,
        p->rec, p->w64, p->b64, err_d);
}

int ensure_workspace(asyrk_problem *p)
{
    if (p->ev[1]) return ASYRK_OK;
    int st;
    const size_t words = (size_t)((p->m + 31) / 32);
    if (!p->xw && (st = dev_alloc(p, (double **)&p->xw, (size_t)p->n)) != ASYRK_OK) return st;
    if (!p->x64 && (st = dev_alloc(p, &p->x64, (size_t)p->n)) != ASYRK_OK) return st;
    if (!p->xt64 && (st = dev_alloc(p, &p->xt64, (size_t)p->n)) != ASYRK_OK) return st;
    if (!p->red_part &&
        (st = dev_alloc(p, &p->red_part, (size_t)ASYRK_MAX_RED_BLOCKS * 4)) != ASYRK_OK)
        return st;
    if (!p->red_count) {
        if ((st = dev_alloc(p, &p->red_count, 1)) != ASYRK_OK) return st;
        ASYRK_CK(cudaMemset(p->red_count, 0, sizeof(unsigned)));
    }
    if (!p->red_out && (st = dev_alloc(p, &p->red_out, 8)) != ASYRK_OK) return st;
    if (!p->busy) {
        if ((st = dev_alloc(p, &p->busy, words)) != ASYRK_OK) return st;
        ASYRK_CK(cudaMemset(p->busy, 0, words * sizeof(unsigned)));
    }
    if (!p->skipped && (st = dev_alloc(p, &p->skipped, 1)) != ASYRK_OK) return st;
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
    cudaFree(p->rec);
    cudaFree(p->col);
    cudaFree(p->val);
    cudaFree(p->b64);
    cudaFree(p->w64);
    cudaFree(p->xw);
    cudaFree(p->x64);
    cudaFree(p->xt64);
    cudaFree(p->g64);
    cudaFree(p->red_part);
    cudaFree(p->red_count);
    cudaFree(p->red_out);
    cudaFree(p->rows_buf);
    cudaFree(p->busy);
    cudaFree(p->skipped);
    if (p->h_out) cudaFreeHost(p->h_out);
    if (p->ev[0]) cudaEventDestroy(p->ev[0]);
    if (p->ev[1]) cudaEventDestroy(p->ev[1]);
    if (cur >= 0 && cur != p->device) cudaSetDevice(cur);
    delete p;
}

static int create_impl(asyrk_problem *p, const int64_t *row_ptr, const int32_t *col_idx,
                       const void *values, const double *b, const asyrk_create_opts *o)
{
    const int64_t m = p->m, n = p->n;
    const bool on_dev = o->device_ptrs != 0;
    cudaStream_t s = (cudaStream_t)o->stream;
    ASYRK_CK(cudaGetDevice(&p->device));
    ASYRK_CK(cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device));

    // 1. row pointers on the host: monotone, no zero rows, padded starts
    std::vector<int64_t> rp((size_t)m + 1);
    if (on_dev)
        ASYRK_CK(cudaMemcpy(rp.data(), row_ptr, (m + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
    else
        memcpy(rp.data(), row_ptr, (m + 1) * sizeof(int64_t));
    if (rp[0] != 0) return set_error(ASYRK_EINVAL, "row_ptr[0] = %lld, expected 0", (long long)rp[0]);
    bool aligned = true;
    int64_t max_len = 0, pad_total = 0;
    std::vector<int64_t> pstart((size_t)m);
    for (int64_t i = 0; i < m; ++i) {
        const int64_t len = rp[i + 1] - rp[i];
        if (len <= 0)
            return set_error(ASYRK_EINVAL, "row %lld is empty or row_ptr decreases (the problem "
                             "has no zero rows)", (long long)i);
        if (rp[i] & 3) aligned = false;
        if (len > max_len) max_len = len;
        pstart[i] = pad_total;
        pad_total += (len + 3) & ~(int64_t)3;
    }
    if (max_len > n) return set_error(ASYRK_EINVAL, "a row has more entries than n");
    if (pad_total != rp[m]) aligned = false;
    p->nnz = rp[m];
    p->nnz_pad = aligned ? p->nnz : pad_total;
    p->max_len = max_len;

    // 2. device arrays
    const size_t es = value_size(p->dtype);
    int st;
    if ((st = dev_alloc(p, &p->rec, (size_t)m)) != ASYRK_OK) return st;
    if ((st = dev_alloc(p, &p->col, (size_t)p->nnz_pad)) != ASYRK_OK) return st;
    if ((st = dev_alloc(p, (char **)&p->val, (size_t)p->nnz_pad * es)) != ASYRK_OK) return st;
    if ((st = dev_alloc(p, &p->b64, (size_t)m)) != ASYRK_OK) return st;
    if ((st = dev_alloc(p, &p->w64, (size_t)m)) != ASYRK_OK) return st;

    // temporaries: the caller's layout on the device (when it is not already)
    int64_t *rp_d = nullptr, *ps_d = nullptr;
    int32_t *col_src = nullptr;
    void *val_src = nullptr;
    double *b_d = nullptr;
    unsigned *err_d = nullptr;
    uint2 *tab_d = nullptr;
    auto cleanup = [&]() {
        cudaFree(rp_d); cudaFree(ps_d); cudaFree(err_d); cudaFree(tab_d);
        if (!on_dev) { cudaFree(b_d); if (!aligned) { cudaFree(col_src); cudaFree(val_src); } }
    };
    auto fail = [&](int code) { cleanup(); return code; };
#define ASYRK_CKC(call)                                                                    \
    do {                                                                                   \
        cudaError_t e__ = (call);                                                          \
        if (e__ != cudaSuccess) return fail(cuda_fail(e__, #call, __FILE__, __LINE__));    \
    } while (0)

    ASYRK_CKC(cudaMalloc((void **)&rp_d, (m + 1) * sizeof(int64_t)));
    ASYRK_CKC(cudaMemcpyAsync(rp_d, rp.data(), (m + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    ASYRK_CKC(cudaMalloc((void **)&err_d, sizeof(unsigned)));
    ASYRK_CKC(cudaMemsetAsync(err_d, 0, sizeof(unsigned), s));
    if (!aligned) {
        ASYRK_CKC(cudaMalloc((void **)&ps_d, m * sizeof(int64_t)));
        ASYRK_CKC(cudaMemcpyAsync(ps_d, pstart.data(), m * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    }
    if (on_dev) {
        col_src = const_cast<int32_t *>(col_idx);
        val_src = const_cast<void *>(values);
        b_d = const_cast<double *>(b);
        if (aligned) {
            ASYRK_CKC(cudaMemcpyAsync(p->col, col_idx, p->nnz * 4, cudaMemcpyDeviceToDevice, s));
            ASYRK_CKC(cudaMemcpyAsync(p->val, values, p->nnz * es, cudaMemcpyDeviceToDevice, s));
        }
    } else {
        if (aligned) {
            col_src = p->col;
            val_src = p->val;
        } else {
            ASYRK_CKC(cudaMalloc((void **)&col_src, p->nnz * 4));
            ASYRK_CKC(cudaMalloc(&val_src, p->nnz * es));
        }
        ASYRK_CKC(cudaMemcpyAsync(col_src, col_idx, p->nnz * 4, cudaMemcpyHostToDevice, s));
        ASYRK_CKC(cudaMemcpyAsync(val_src, values, p->nnz * es, cudaMemcpyHostToDevice, s));
        ASYRK_CKC(cudaMalloc((void **)&b_d, m * sizeof(double)));
        ASYRK_CKC(cudaMemcpyAsync(b_d, b, m * sizeof(double), cudaMemcpyHostToDevice, s));
    }
    // with aligned input the row pass reads the final arrays in place
    const int32_t *rs_col = aligned ? p->col : col_src;
    const void *rs_val = aligned ? p->val : val_src;
    switch (p->dtype) {
    case ASYRK_F64: launch_row_setup<double>(p, rp_d, ps_d, rs_col, rs_val, b_d, err_d, s); break;
    case ASYRK_F32: launch_row_setup<float>(p, rp_d, ps_d, rs_col, rs_val, b_d, err_d, s); break;
    default: launch_row_setup<bf16_t>(p, rp_d, ps_d, rs_col, rs_val, b_d, err_d, s); break;
    }
    ASYRK_CKC(cudaGetLastError());
    unsigned err_h = 0;
    ASYRK_CKC(cudaMemcpyAsync(&err_h, err_d, sizeof err_h, cudaMemcpyDeviceToHost, s));
    std::vector<double> w((size_t)m), bh((size_t)m);
    ASYRK_CKC(cudaMemcpyAsync(w.data(), p->w64, m * sizeof(double), cudaMemcpyDeviceToHost, s));
    ASYRK_CKC(cudaMemcpyAsync(bh.data(), p->b64, m * sizeof(double), cudaMemcpyDeviceToHost, s));
    ASYRK_CKC(cudaStreamSynchronize(s));
    if (err_h) {
        const char *why = (err_h & ERR_COL_RANGE)  ? "a column index is outside [0, n)"
                          : (err_h & ERR_COL_ORDER) ? "columns are not strictly ascending within a row"
                          : (err_h & ERR_VAL)       ? "a value is not finite"
                          : (err_h & ERR_ZERO_ROW)  ? "a row has zero norm (the problem has no zero rows)"
                                                    : "b has a non-finite entry";
        return fail(set_error(ASYRK_EINVAL, "malformed problem: %s", why));
    }

    // 3. alias table of the row weights
    double F = 0.0, bb = 0.0;
    for (int64_t i = 0; i < m; ++i) F += w[(size_t)i];
    for (int64_t i = 0; i < m; ++i) bb += bh[(size_t)i] * bh[(size_t)i];
    if (!(F > 0.0) || !isfinite(F)) return fail(set_error(ASYRK_EINVAL, "||A||_F^2 is not finite"));
    p->frob2 = F;
    p->bnorm = sqrt(bb);
    std::vector<uint2> tab;
    p->uniform = build_alias(w, F, tab) ? 1 : 0;
    if (!p->uniform) {
        ASYRK_CKC(cudaMalloc((void **)&tab_d, m * sizeof(uint2)));
        ASYRK_CKC(cudaMemcpyAsync(tab_d, tab.data(), m * sizeof(uint2), cudaMemcpyHostToDevice, s));
        k_set_alias<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(m, tab_d, p->rec);
        ASYRK_CKC(cudaGetLastError());
    }
    ASYRK_CKC(cudaStreamSynchronize(s));
    cleanup();
#undef ASYRK_CKC
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
        cudaFree(p->rows_buf);
        p->rows_buf = nullptr;
        p->rows_cap = 0;
        ASYRK_CK(cudaMalloc((void **)&p->rows_buf, count * sizeof(int32_t)));
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
