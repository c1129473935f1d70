// lsq.cu -- least squares through a square consistent system (Section 6).
//
// min ||A x - b|| is solved by the method applied to
//     [ 0   phi A^T ] [x]   [phi A^T b]
//     [ A   -zeta I ] [y] = [    0    ]
// whose solutions have x = zeta x_LS and y = A x_LS.  Rows, in order: one per
// non-empty column j of A (entries (n + i, phi A_ij), i ascending; right side
// phi * sum_i A_ij b_i summed in ascending i in FP64 without fused
// multiply-adds); then one per row i of A (its entries, then (n + i, -zeta);
// right side 0).  A column of zeros would give the row 0 = 0 and is left out.
//
// The system is assembled on the GPU: a stable LSD radix sort of the entries
// by column gives A^T in CSR with rows ascending inside each column, two
// fills write the two blocks, and the result goes through asyrk_create.
#include <math.h>
#include <string.h>

#include <vector>

#include "common.cuh"
#include "scan.cuh"

namespace asyrk {

namespace {

constexpr int SORT_THREADS = 256;
constexpr int SORT_ITEMS = 8;  // keys per thread; a warp owns 8 rounds of 32 consecutive keys
constexpr int SORT_TILE = SORT_THREADS * SORT_ITEMS;
constexpr int SORT_WARPS = SORT_THREADS / 32;

__device__ __forceinline__ double widen_v(double v) { return v; }
__device__ __forceinline__ double widen_v(float v) { return (double)v; }
__device__ __forceinline__ double widen_v(bf16_t v)
{
    return (double)__uint_as_float(((unsigned)v.bits) << 16);
}
__device__ __forceinline__ void narrow_v(double d, double &v) { v = d; }
__device__ __forceinline__ void narrow_v(double d, float &v) { v = (float)d; }
__device__ __forceinline__ void narrow_v(double d, bf16_t &v)
{
    // round to nearest even from FP32 (the FP64 value is first rounded to FP32)
    const unsigned u = __float_as_uint((float)d);
    v.bits = (unsigned short)((u + 0x7fffu + ((u >> 16) & 1u)) >> 16);
}

enum : unsigned { BAD_COL = 1u, BAD_ORDER = 2u, BAD_VAL = 4u, BAD_B = 8u };

// ---- stable LSD radix sort of (key, value) by 8-bit digits ----------------
// Tile t holds keys [t*SORT_TILE, (t+1)*SORT_TILE); inside it warp w holds
// SORT_ITEMS rounds of 32 consecutive keys starting at w*32*SORT_ITEMS, so
// (warp, round, lane) is the input order and the scatter keeps it.
__global__ void __launch_bounds__(SORT_THREADS) k_radix_hist(const uint32_t *__restrict__ keys,
                                                            int64_t count, int shift,
                                                            int64_t *__restrict__ hist,
                                                            int64_t tiles)
{
    __shared__ unsigned h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * SORT_TILE;
    for (int k = threadIdx.x; k < SORT_TILE; k += SORT_THREADS) {
        const int64_t q = base + k;
        if (q < count) atomicAdd(&h[(keys[q] >> shift) & 255u], 1u);
    }
    __syncthreads();
    // digit-major, so one exclusive scan gives every (digit, tile) its offset
    hist[(int64_t)threadIdx.x * tiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(SORT_THREADS) k_radix_scatter(
    const uint32_t *__restrict__ keys, const uint32_t *__restrict__ vals, int64_t count, int shift,
    const int64_t *__restrict__ offs, int64_t tiles, uint32_t *__restrict__ keys_out,
    uint32_t *__restrict__ vals_out)
{
    __shared__ unsigned wcnt[SORT_WARPS][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = lane; d < 256; d += 32) wcnt[w][d] = 0;
    __syncwarp();
    const int64_t base = (int64_t)blockIdx.x * SORT_TILE + (int64_t)w * 32 * SORT_ITEMS;
    const unsigned lt = (1u << lane) - 1u;
    uint32_t k_[SORT_ITEMS], v_[SORT_ITEMS];
    unsigned rank[SORT_ITEMS];
    int dig[SORT_ITEMS];
#pragma unroll
    for (int r = 0; r < SORT_ITEMS; ++r) {
        const int64_t q = base + r * 32 + lane;
        const bool in = q < count;
        k_[r] = in ? keys[q] : 0u;
        v_[r] = in ? vals[q] : 0u;
        dig[r] = in ? (int)((k_[r] >> shift) & 255u) : 256;  // 256: no key
        const unsigned peers = __match_any_sync(0xffffffffu, dig[r]);
        const unsigned before = (in ? wcnt[w][dig[r]] : 0u);
        rank[r] = before + __popc(peers & lt);
        __syncwarp();
        if (in && (peers & lt) == 0) wcnt[w][dig[r]] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {  // per digit: exclusive scan over the warps
        const int d = threadIdx.x;
        unsigned run = 0;
        for (int ww = 0; ww < SORT_WARPS; ++ww) {
            const unsigned c = wcnt[ww][d];
            wcnt[ww][d] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < SORT_ITEMS; ++r) {
        if (dig[r] == 256) continue;
        const int64_t pos = offs[(int64_t)dig[r] * tiles + blockIdx.x] + wcnt[w][dig[r]] + rank[r];
        keys_out[pos] = k_[r];
        vals_out[pos] = v_[r];
    }
}

// ---- the system's pieces ------------------------------------------------
// One thread per row of A: checks, the entry -> row map, column counts.
template <typename VT>
__global__ void k_lsq_rows(int64_t m, int64_t n, const int64_t *__restrict__ rp,
                           const int32_t *__restrict__ col, const VT *__restrict__ val,
                           const double *__restrict__ b, uint32_t *__restrict__ row_of,
                           int64_t *__restrict__ ccount, unsigned *__restrict__ err)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    unsigned bad = 0;
    int32_t prev = -1;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
        const int32_t c = col[k];
        if (c < 0 || (int64_t)c >= n) {
            bad |= BAD_COL;
            continue;
        }
        if (c <= prev) bad |= BAD_ORDER;
        prev = c;
        if (!isfinite(widen_v(val[k]))) bad |= BAD_VAL;
        row_of[k] = (uint32_t)i;
        atomicAdd((unsigned long long *)&ccount[c], 1ull);
    }
    if (b && !isfinite(b[i])) bad |= BAD_B;
    if (bad) atomicOr(err, bad);
}

__global__ void k_iota_u32(uint32_t *__restrict__ v, int64_t count)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < count) v[q] = (uint32_t)q;
}

__global__ void k_nonempty(const int64_t *__restrict__ ccount, int64_t n, int64_t *__restrict__ flag)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) flag[j] = ccount[j] > 0 ? 1 : 0;
}

// A^T block: sorted position p holds entry k = perm[p] of column j = key[p].
template <typename VT>
__global__ void k_lsq_first_block(int64_t nnz, int64_t n, const uint32_t *__restrict__ perm,
                                  const uint32_t *__restrict__ row_of, const VT *__restrict__ val,
                                  double phi, int32_t *__restrict__ acol, VT *__restrict__ aval)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nnz) return;
    const uint32_t k = perm[p];
    acol[p] = (int32_t)(n + row_of[k]);
    VT v;
    if (phi == 1.0) {
        v = val[k];
    } else {
        narrow_v(__dmul_rn(phi, widen_v(val[k])), v);
    }
    aval[p] = v;
}

// One thread per column: its row's start and phi * (A^T b)_j in ascending i.
template <typename VT>
__global__ void k_lsq_rhs(int64_t n, const int64_t *__restrict__ ccount,
                          const int64_t *__restrict__ cstart, const int64_t *__restrict__ rowidx,
                          const uint32_t *__restrict__ perm, const uint32_t *__restrict__ row_of,
                          const VT *__restrict__ val, const double *__restrict__ b, double phi,
                          int64_t *__restrict__ arp, double *__restrict__ ab)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n || ccount[j] == 0) return;
    double s = 0.0;
    for (int64_t p = cstart[j]; p < cstart[j] + ccount[j]; ++p) {
        const uint32_t k = perm[p];
        s = __dadd_rn(s, __dmul_rn(widen_v(val[k]), b[row_of[k]]));
    }
    const int64_t r = rowidx[j];
    arp[r] = cstart[j];
    ab[r] = __dmul_rn(phi, s);
}

// One thread per row i of A: row nne + i of the system, [a_i, -zeta e_i].
template <typename VT>
__global__ void k_lsq_second_block(int64_t m, int64_t n, int64_t nne, int64_t nnz,
                                   const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                                   const VT *__restrict__ val, double zeta,
                                   int64_t *__restrict__ arp, int32_t *__restrict__ acol,
                                   VT *__restrict__ aval, double *__restrict__ ab)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    int64_t d = nnz + rp[i] + i;
    arp[nne + i] = d;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k, ++d) {
        acol[d] = col[k];
        aval[d] = val[k];
    }
    acol[d] = (int32_t)(n + i);
    VT z;
    narrow_v(-zeta, z);
    aval[d] = z;
    ab[nne + i] = 0.0;
    if (i == m - 1) arp[nne + m] = d + 1;
}

__global__ void k_lsq_extract(const double *__restrict__ z, int64_t n, double zeta,
                              double *__restrict__ x)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) x[j] = __ddiv_rn(z[j], zeta);
}

inline unsigned grid_for(int64_t count, int threads = 256)
{
    return (unsigned)((count + threads - 1) / threads);
}

// device buffers freed on every exit path
struct DevTmp {
    std::vector<void *> ptrs;
    template <typename T>
    int alloc(T **p, size_t count)
    {
        *p = nullptr;
        cudaError_t e = cudaMalloc((void **)p, (count ? count : 1) * sizeof(T));
        if (e != cudaSuccess) {
            *p = nullptr;
            (void)cudaGetLastError();
            return set_error(e == cudaErrorMemoryAllocation ? ASYRK_ENOMEM : ASYRK_ECUDA,
                             "cudaMalloc of %zu bytes failed: %s", count * sizeof(T),
                             cudaGetErrorString(e));
        }
        ptrs.push_back((void *)*p);
        return ASYRK_OK;
    }
    ~DevTmp()
    {
        for (void *q : ptrs) cudaFree(q);
    }
};

size_t dtype_size(int dtype)
{
    return dtype == ASYRK_F64 ? 8 : dtype == ASYRK_F32 ? 4 : 2;
}

// v as the system stores it (the host twin of narrow_v): x = zeta_s x_LS holds
// for the stored zeta_s, so the solution is read back with that value.
double stored_value(int dtype, double v)
{
    if (dtype == ASYRK_F64) return v;
    const float f = (float)v;
    if (dtype == ASYRK_F32) return (double)f;
    uint32_t u;
    memcpy(&u, &f, 4);
    u = ((u + 0x7fffu + ((u >> 16) & 1u)) >> 16) << 16;
    float g;
    memcpy(&g, &u, 4);
    return (double)g;
}

}  // namespace

// ---- Lanczos on A^T A (the estimate of sigma_r for zeta) -----------------
__global__ void k_rand_sign(double *__restrict__ u, int64_t m, uint2 key)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const uint4 r = philox4x32_10(make_uint4((unsigned)i, (unsigned)(i >> 32), 0x4c414eu, 2u), key);
    u[i] = (r.x & 1u) ? 1.0 : -1.0;
}

template <typename VT>
__global__ void k_spmv(int64_t m, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                       const VT *__restrict__ val, const double *__restrict__ v,
                       double *__restrict__ y)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    double s = 0.0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) s += widen_v(val[k]) * v[col[k]];
    y[i] = s;
}

// w += A^T y (w zeroed by the caller); FP64 atomics, so the rounding order varies
template <typename VT>
__global__ void k_spmv_t(int64_t m, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                         const VT *__restrict__ val, const double *__restrict__ y,
                         double *__restrict__ w)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const double yi = y[i];
    if (yi == 0.0) return;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) atomicAdd(&w[col[k]], widen_v(val[k]) * yi);
}

// out[j] = Q[:, j] . w for j < ncols (one block per column, fixed reduction order)
__global__ void k_dot_cols(const double *__restrict__ Q, int64_t ld, const double *__restrict__ w,
                           int64_t n, double *__restrict__ out)
{
    __shared__ double part[256];
    const double *q = Q + (int64_t)blockIdx.x * ld;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += 256) s += q[i] * w[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = part[0];
}

// w -= Q[:, 0:ncols] h
__global__ void k_sub_cols(double *__restrict__ w, const double *__restrict__ Q, int64_t ld,
                           int ncols, const double *__restrict__ h, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = w[i];
    for (int j = 0; j < ncols; ++j) s -= Q[(int64_t)j * ld + i] * h[j];
    w[i] = s;
}

__global__ void k_axpy_d(double *__restrict__ y, const double *__restrict__ x, double a, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] += a * x[i];
}

__global__ void k_scale_d(double *__restrict__ y, const double *__restrict__ x, double a, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = a * x[i];
}

// number of eigenvalues below x of the symmetric tridiagonal (a, b), b[0] unused
static int sturm_count(const std::vector<double> &a, const std::vector<double> &b, double x)
{
    int c = 0;
    double d = 1.0;
    for (size_t i = 0; i < a.size(); ++i) {
        d = a[i] - x - (i ? b[i] * b[i] / d : 0.0);
        if (d == 0.0) d = -1e-300;
        if (d < 0.0) ++c;
    }
    return c;
}

// the k-th smallest eigenvalue (k from 1) by bisection on the Sturm count
static double tridiag_eig(const std::vector<double> &a, const std::vector<double> &b, int k)
{
    double lo = a[0], hi = a[0];
    for (size_t i = 0; i < a.size(); ++i) {  // Gershgorin
        const double r = (i ? fabs(b[i]) : 0.0) + (i + 1 < a.size() ? fabs(b[i + 1]) : 0.0);
        lo = fmin(lo, a[i] - r);
        hi = fmax(hi, a[i] + r);
    }
    for (int it = 0; it < 200 && hi - lo > 1e-15 * fmax(fabs(lo), fabs(hi)); ++it) {
        const double mid = 0.5 * (lo + hi);
        if (sturm_count(a, b, mid) >= k) hi = mid; else lo = mid;
    }
    return 0.5 * (lo + hi);
}

// Extreme Ritz values of A^T A after `steps` Lanczos steps with full
// reorthogonalisation (twice per step), started from A^T u so that the Krylov
// space stays in the row space of A: lmin estimates the smallest NONZERO
// eigenvalue (Ritz values under 1e-10 lmax are rounding-level null-space
// components and are passed over).
template <typename VT>
static int lanczos_extremes(int64_t m, int64_t n, const int64_t *rp, const int32_t *col, const VT *val,
                     int steps, uint64_t seed, cudaStream_t s, double *lmin, double *lmax)
{
    if (steps > n) steps = (int)n;
    DevTmp t;
    double *Q, *u, *y, *w, *h;
    int st;
    if ((st = t.alloc(&Q, (size_t)n * (steps + 1))) || (st = t.alloc(&u, (size_t)m)) ||
        (st = t.alloc(&y, (size_t)m)) || (st = t.alloc(&w, (size_t)n)) ||
        (st = t.alloc(&h, (size_t)steps + 1)))
        return st;
    double hb[2];
    auto fetch = [&](int count) -> int {
        ASYRK_CK(cudaMemcpyAsync(hb, h, count * sizeof(double), cudaMemcpyDeviceToHost, s));
        ASYRK_CK(cudaStreamSynchronize(s));
        return ASYRK_OK;
    };
    const uint2 key = make_uint2((unsigned)seed, (unsigned)(seed >> 32));
    k_rand_sign<<<grid_for(m), 256, 0, s>>>(u, m, key);
    ASYRK_CK(cudaMemsetAsync(w, 0, n * sizeof(double), s));
    k_spmv_t<VT><<<grid_for(m), 256, 0, s>>>(m, rp, col, val, u, w);
    k_dot_cols<<<1, 256, 0, s>>>(w, n, w, n, h);
    ASYRK_CK(cudaGetLastError());
    if ((st = fetch(1)) != ASYRK_OK) return st;
    double beta = sqrt(hb[0]);
    if (!(beta > 0.0)) return set_error(ASYRK_EINVAL, "A^T u = 0: the matrix has no nonzero entry");
    k_scale_d<<<grid_for(n), 256, 0, s>>>(Q, w, 1.0 / beta, n);
    std::vector<double> al, be(1, 0.0);
    for (int j = 0; j < steps; ++j) {
        double *qj = Q + (int64_t)j * n;
        k_spmv<VT><<<grid_for(m), 256, 0, s>>>(m, rp, col, val, qj, y);
        ASYRK_CK(cudaMemsetAsync(w, 0, n * sizeof(double), s));
        k_spmv_t<VT><<<grid_for(m), 256, 0, s>>>(m, rp, col, val, y, w);
        if (j > 0) k_axpy_d<<<grid_for(n), 256, 0, s>>>(w, qj - n, -be[j], n);
        k_dot_cols<<<1, 256, 0, s>>>(qj, n, w, n, h);
        ASYRK_CK(cudaGetLastError());
        if ((st = fetch(1)) != ASYRK_OK) return st;
        const double alpha = hb[0];
        k_axpy_d<<<grid_for(n), 256, 0, s>>>(w, qj, -alpha, n);
        for (int pass = 0; pass < 2; ++pass) {
            k_dot_cols<<<j + 1, 256, 0, s>>>(Q, n, w, n, h);
            k_sub_cols<<<grid_for(n), 256, 0, s>>>(w, Q, n, j + 1, h, n);
        }
        k_dot_cols<<<1, 256, 0, s>>>(w, n, w, n, h);
        ASYRK_CK(cudaGetLastError());
        if ((st = fetch(1)) != ASYRK_OK) return st;
        al.push_back(alpha);
        double amax = 0.0;
        for (double a : al) amax = fmax(amax, fabs(a));
        beta = sqrt(hb[0]);
        if (!(beta > 1e-12 * amax) || j + 1 == steps) break;
        be.push_back(beta);
        k_scale_d<<<grid_for(n), 256, 0, s>>>(Q + (int64_t)(j + 1) * n, w, 1.0 / beta, n);
    }
    be.resize(al.size());
    const int k = (int)al.size();
    *lmax = tridiag_eig(al, be, k);
    const int c0 = sturm_count(al, be, 1e-10 * *lmax);
    if (c0 >= k) return set_error(ASYRK_EINVAL, "no nonzero Ritz value");
    *lmin = tridiag_eig(al, be, c0 + 1);
    return ASYRK_OK;
}


// A CSR matrix (and optionally b) on the device, copied there when the
// caller's arrays are host arrays; row_ptr checked on the host.
struct Csr {
    int64_t m = 0, n = 0, nnz = 0;
    const int64_t *rp = nullptr;
    const int32_t *col = nullptr;
    const void *val = nullptr;
    const double *b = nullptr;
};

static int stage_csr(int64_t m, int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                     const void *values, int vdtype, const double *b, bool on_dev, cudaStream_t s,
                     DevTmp &t, Csr &c)
{
    std::vector<int64_t> rp((size_t)m + 1);
    if (on_dev)
        ASYRK_CK(cudaMemcpy(rp.data(), row_ptr, (m + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
    else
        memcpy(rp.data(), row_ptr, (m + 1) * sizeof(int64_t));
    if (rp[0] != 0) return set_error(ASYRK_EINVAL, "row_ptr[0] must be 0");
    for (int64_t i = 0; i < m; ++i)
        if (rp[i + 1] < rp[i] || rp[i + 1] - rp[i] > n)
            return set_error(ASYRK_EINVAL, "row_ptr decreases or row %lld is longer than n",
                             (long long)i);
    c.m = m;
    c.n = n;
    c.nnz = rp[m];
    if (c.nnz > 0xffffffffLL) return set_error(ASYRK_EINVAL, "more than 2^32-1 nonzeros");
    c.rp = row_ptr;
    c.col = col_idx;
    c.val = values;
    c.b = b;
    if (on_dev) return ASYRK_OK;
    const size_t es = dtype_size(vdtype);
    int64_t *a;
    int32_t *cc;
    char *v;
    double *bb = nullptr;
    int st;
    if ((st = t.alloc(&a, (size_t)m + 1)) || (st = t.alloc(&cc, (size_t)c.nnz)) ||
        (st = t.alloc(&v, (size_t)c.nnz * es)) || (b && (st = t.alloc(&bb, (size_t)m))))
        return st;
    ASYRK_CK(cudaMemcpyAsync(a, rp.data(), (m + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    ASYRK_CK(cudaMemcpyAsync(cc, col_idx, c.nnz * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    ASYRK_CK(cudaMemcpyAsync(v, values, c.nnz * es, cudaMemcpyHostToDevice, s));
    if (b) ASYRK_CK(cudaMemcpyAsync(bb, b, m * sizeof(double), cudaMemcpyHostToDevice, s));
    c.rp = a;
    c.col = cc;
    c.val = v;
    c.b = bb;
    return ASYRK_OK;
}

// Column range and order, finite values and b; fills the entry -> row map and
// the column counts.
template <typename VT>
static int check_rows(const Csr &c, uint32_t *row_of, int64_t *ccount, unsigned *err,
                      cudaStream_t s)
{
    ASYRK_CK(cudaMemsetAsync(ccount, 0, c.n * sizeof(int64_t), s));
    ASYRK_CK(cudaMemsetAsync(err, 0, sizeof(unsigned), s));
    k_lsq_rows<VT><<<grid_for(c.m), 256, 0, s>>>(c.m, c.n, c.rp, c.col, (const VT *)c.val, c.b,
                                                 row_of, ccount, err);
    ASYRK_CK(cudaGetLastError());
    unsigned bad = 0;
    ASYRK_CK(cudaMemcpyAsync(&bad, err, sizeof bad, cudaMemcpyDeviceToHost, s));
    ASYRK_CK(cudaStreamSynchronize(s));
    if (bad & BAD_COL) return set_error(ASYRK_EINVAL, "a column index is outside [0, n)");
    if (bad & BAD_ORDER) return set_error(ASYRK_EINVAL, "column indices not strictly ascending in a row");
    if (bad & BAD_VAL) return set_error(ASYRK_EINVAL, "a value is not finite");
    if (bad & BAD_B) return set_error(ASYRK_EINVAL, "b is not finite");
    return ASYRK_OK;
}

constexpr int DEFAULT_LANCZOS_STEPS = 100;

template <typename VT>
static int lsq_build(asyrk_problem **out, const Csr &c, int vdtype, const asyrk_lsq_opts &o,
                     cudaStream_t s)
{
    const int64_t m = c.m, n = c.n, nnz = c.nnz;
    const VT *val = (const VT *)c.val;
    const double phi = o.phi == 0.0 ? 1.0 : o.phi;
    DevTmp t;
    int st;
    uint32_t *row_of, *keys[2], *perm[2];
    int64_t *ccount, *cstart, *flag, *rowidx, *hist, *offs, *scan_tmp, *totals;
    unsigned *err;
    const int64_t tiles = (nnz + SORT_TILE - 1) / SORT_TILE;
    const int64_t scan_max = (256 * tiles > n ? 256 * tiles : n);
    if ((st = t.alloc(&row_of, (size_t)nnz)) || (st = t.alloc(&keys[0], (size_t)nnz)) ||
        (st = t.alloc(&keys[1], (size_t)nnz)) || (st = t.alloc(&perm[0], (size_t)nnz)) ||
        (st = t.alloc(&perm[1], (size_t)nnz)) || (st = t.alloc(&ccount, (size_t)n)) ||
        (st = t.alloc(&cstart, (size_t)n)) || (st = t.alloc(&flag, (size_t)n)) ||
        (st = t.alloc(&rowidx, (size_t)n)) || (st = t.alloc(&hist, (size_t)(256 * tiles))) ||
        (st = t.alloc(&offs, (size_t)(256 * tiles))) ||
        (st = t.alloc(&scan_tmp, (size_t)scan_tmp_count(scan_max))) ||
        (st = t.alloc(&totals, 2)) || (st = t.alloc(&err, 1)))
        return st;

    // 1. checks, entry -> row map, column counts
    if ((st = check_rows<VT>(c, row_of, ccount, err, s)) != ASYRK_OK) return st;

    // 2. zeta: the caller's, or Section 6's sigma_r / sqrt(2) with sigma_r^2 the
    //    smallest nonzero Ritz value of A^T A
    double zeta = o.zeta;
    if (zeta == 0.0) {
        double lmin = 0.0, lmax = 0.0;
        const int steps = o.lanczos_steps > 0 ? o.lanczos_steps : DEFAULT_LANCZOS_STEPS;
        if ((st = lanczos_extremes<VT>(m, n, c.rp, c.col, val, steps, o.seed, s, &lmin, &lmax)) !=
            ASYRK_OK)
            return st;
        zeta = sqrt(0.5 * lmin);
    }

    // 3. entries sorted by column, stable, so rows ascend inside each column
    int cur = 0;
    if (nnz > 0) {
        ASYRK_CK(cudaMemcpyAsync(keys[0], c.col, nnz * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
        k_iota_u32<<<grid_for(nnz), 256, 0, s>>>(perm[0], nnz);
        ASYRK_CK(cudaGetLastError());
        int bits = 0;
        while (bits < 32 && ((uint64_t)(n - 1) >> bits) != 0) ++bits;
        for (int shift = 0; shift < bits; shift += 8) {
            k_radix_hist<<<(unsigned)tiles, SORT_THREADS, 0, s>>>(keys[cur], nnz, shift, hist, tiles);
            ASYRK_CK(cudaGetLastError());
            if ((st = exclusive_scan(hist, offs, 256 * tiles, scan_tmp, totals, s)) != ASYRK_OK)
                return st;
            k_radix_scatter<<<(unsigned)tiles, SORT_THREADS, 0, s>>>(
                keys[cur], perm[cur], nnz, shift, offs, tiles, keys[cur ^ 1], perm[cur ^ 1]);
            ASYRK_CK(cudaGetLastError());
            cur ^= 1;
        }
    }

    // 4. column starts and the row number of each non-empty column
    if ((st = exclusive_scan(ccount, cstart, n, scan_tmp, totals, s)) != ASYRK_OK) return st;
    k_nonempty<<<grid_for(n), 256, 0, s>>>(ccount, n, flag);
    ASYRK_CK(cudaGetLastError());
    if ((st = exclusive_scan(flag, rowidx, n, scan_tmp, totals + 1, s)) != ASYRK_OK) return st;
    int64_t nne = 0;
    ASYRK_CK(cudaMemcpyAsync(&nne, totals + 1, sizeof nne, cudaMemcpyDeviceToHost, s));
    ASYRK_CK(cudaStreamSynchronize(s));

    // 5. the system
    const int64_t rows = nne + m, annz = 2 * nnz + m;
    int64_t *arp;
    int32_t *acol;
    VT *aval;
    double *ab;
    if ((st = t.alloc(&arp, (size_t)rows + 1)) || (st = t.alloc(&acol, (size_t)annz)) ||
        (st = t.alloc(&aval, (size_t)annz)) || (st = t.alloc(&ab, (size_t)rows)))
        return st;
    if (nnz > 0) {
        k_lsq_first_block<VT><<<grid_for(nnz), 256, 0, s>>>(nnz, n, perm[cur], row_of, val, phi,
                                                            acol, aval);
        k_lsq_rhs<VT><<<grid_for(n), 256, 0, s>>>(n, ccount, cstart, rowidx, perm[cur], row_of,
                                                  val, c.b, phi, arp, ab);
    }
    k_lsq_second_block<VT><<<grid_for(m), 256, 0, s>>>(m, n, nne, nnz, c.rp, c.col, val, zeta, arp,
                                                       acol, aval, ab);
    ASYRK_CK(cudaGetLastError());
    ASYRK_CK(cudaStreamSynchronize(s));

    asyrk_create_opts co;
    memset(&co, 0, sizeof co);
    co.seed = o.seed;
    co.device_ptrs = 1;
    co.stream = o.stream;
    asyrk_problem *p = nullptr;
    if ((st = asyrk_create(&p, rows, n + m, arp, acol, aval, vdtype, ab, &co)) != ASYRK_OK) return st;
    p->lsq_n = n;
    p->lsq_zeta = stored_value(vdtype, zeta);
    p->lsq_phi = phi;
    *out = p;
    return ASYRK_OK;
}

template <typename VT>
static int spectrum_impl(const Csr &c, int steps, uint64_t seed, cudaStream_t s, double *lmin,
                         double *lmax)
{
    DevTmp t;
    uint32_t *row_of;
    int64_t *ccount;
    unsigned *err;
    int st;
    if ((st = t.alloc(&row_of, (size_t)c.nnz)) || (st = t.alloc(&ccount, (size_t)c.n)) ||
        (st = t.alloc(&err, 1)))
        return st;
    if ((st = check_rows<VT>(c, row_of, ccount, err, s)) != ASYRK_OK) return st;
    return lanczos_extremes<VT>(c.m, c.n, c.rp, c.col, (const VT *)c.val, steps, seed, s, lmin, lmax);
}

}  // namespace asyrk

using namespace asyrk;

static int check_dims(int64_t m, int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                      const void *values, int vdtype)
{
    if (m <= 0 || n <= 0 || m + n > 0x7fffffffLL)
        return set_error(ASYRK_EINVAL, "m, n >= 1 and m + n <= 2^31-1 required");
    if (!row_ptr || !col_idx || !values) return set_error(ASYRK_EINVAL, "NULL array");
    if (vdtype != ASYRK_F64 && vdtype != ASYRK_F32 && vdtype != ASYRK_BF16)
        return set_error(ASYRK_EINVAL, "unknown value dtype %d", vdtype);
    return ASYRK_OK;
}

extern "C" int asyrk_lsq_create(asyrk_problem **out, int64_t m, int64_t n, const int64_t *row_ptr,
                                const int32_t *col_idx, const void *values, int vdtype,
                                const double *b, const asyrk_lsq_opts *opts)
{
    if (!out) return set_error(ASYRK_EINVAL, "out is NULL");
    *out = nullptr;
    if (!opts) return set_error(ASYRK_EINVAL, "opts is NULL");
    const asyrk_lsq_opts o = *opts;
    int st = check_dims(m, n, row_ptr, col_idx, values, vdtype);
    if (st != ASYRK_OK) return st;
    if (!b) return set_error(ASYRK_EINVAL, "NULL b");
    if (o.zeta < 0.0 || !isfinite(o.zeta)) return set_error(ASYRK_EINVAL, "zeta must be > 0 (0: estimated)");
    if (o.phi < 0.0 || !isfinite(o.phi)) return set_error(ASYRK_EINVAL, "phi must be > 0 (0: 1)");
    if (o.lanczos_steps < 0) return set_error(ASYRK_EINVAL, "lanczos_steps < 0");
    cudaStream_t s = (cudaStream_t)o.stream;
    DevTmp t;
    Csr c;
    if ((st = stage_csr(m, n, row_ptr, col_idx, values, vdtype, b, o.device_ptrs != 0, s, t, c)) !=
        ASYRK_OK)
        return st;
    switch (vdtype) {
    case ASYRK_F64: return lsq_build<double>(out, c, vdtype, o, s);
    case ASYRK_F32: return lsq_build<float>(out, c, vdtype, o, s);
    default: return lsq_build<bf16_t>(out, c, vdtype, o, s);
    }
}

extern "C" int asyrk_lsq_params(const asyrk_problem *p, double *zeta, double *phi)
{
    if (!p) return set_error(ASYRK_EINVAL, "NULL problem");
    if (p->lsq_n <= 0) return set_error(ASYRK_EINVAL, "not a least-squares problem");
    if (zeta) *zeta = p->lsq_zeta;
    if (phi) *phi = p->lsq_phi;
    return ASYRK_OK;
}

extern "C" int asyrk_spectrum_estimate(int64_t m, int64_t n, const int64_t *row_ptr,
                                       const int32_t *col_idx, const void *values, int vdtype,
                                       int device_ptrs, int32_t steps, uint64_t seed,
                                       void *stream, double *lambda_min, double *lambda_max)
{
    int st = check_dims(m, n, row_ptr, col_idx, values, vdtype);
    if (st != ASYRK_OK) return st;
    if (!lambda_min || !lambda_max) return set_error(ASYRK_EINVAL, "NULL output");
    if (steps < 0) return set_error(ASYRK_EINVAL, "steps < 0");
    if (steps == 0) steps = DEFAULT_LANCZOS_STEPS;
    cudaStream_t s = (cudaStream_t)stream;
    DevTmp t;
    Csr c;
    if ((st = stage_csr(m, n, row_ptr, col_idx, values, vdtype, nullptr, device_ptrs != 0, s, t,
                        c)) != ASYRK_OK)
        return st;
    switch (vdtype) {
    case ASYRK_F64: return spectrum_impl<double>(c, steps, seed, s, lambda_min, lambda_max);
    case ASYRK_F32: return spectrum_impl<float>(c, steps, seed, s, lambda_min, lambda_max);
    default: return spectrum_impl<bf16_t>(c, steps, seed, s, lambda_min, lambda_max);
    }
}

extern "C" int asyrk_lsq_solution(asyrk_problem *p, const double *z, int on_device, double *x_ls)
{
    if (!p || !z || !x_ls) return set_error(ASYRK_EINVAL, "NULL argument");
    if (p->lsq_n <= 0) return set_error(ASYRK_EINVAL, "not a least-squares problem");
    const int64_t n = p->lsq_n;
    if (on_device) {
        k_lsq_extract<<<grid_for(n), 256>>>(z, n, p->lsq_zeta, x_ls);
        ASYRK_CK(cudaGetLastError());
        ASYRK_CK(cudaDeviceSynchronize());
        return ASYRK_OK;
    }
    DevTmp t;
    double *zd, *xd;
    int st;
    if ((st = t.alloc(&zd, (size_t)n)) || (st = t.alloc(&xd, (size_t)n))) return st;
    ASYRK_CK(cudaMemcpy(zd, z, n * sizeof(double), cudaMemcpyHostToDevice));
    k_lsq_extract<<<grid_for(n), 256>>>(zd, n, p->lsq_zeta, xd);
    ASYRK_CK(cudaGetLastError());
    ASYRK_CK(cudaMemcpy(x_ls, xd, n * sizeof(double), cudaMemcpyDeviceToHost));
    return ASYRK_OK;
}
