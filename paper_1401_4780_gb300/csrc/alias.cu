// alias.cu -- ||A||_F^2, ||b||^2 and the alias table of the row weights, on the GPU.
//
// Rows are drawn with probability w_i / F (w_i = ||a_i||^2, F = ||A||_F^2,
// Section 1) through Walker's alias table.  The table is defined by one
// sequential sweep (the header of asyrk.h states it); this file evaluates the
// same table in parallel:
//   * F sums blocks of 2048 consecutive w_i in index order, then the block sums
//     in order (the same order as the definition, so the same FP64 value);
//   * integer masses M_i = floor(((w_i m) / F) 2^32), corrected so that they add
//     up to m U exactly (U = 2^32, one bucket);
//   * lights (M < U) and heavies (M >= U) are compacted in index order by one
//     prefix sum; S_k = deficit U - M of the lights before light k, C_t = excess
//     M - U of heavies 0..t (prefix sums of exact integers);
//   * light k pairs with heavy #{t : C_t < S_k} (a binary search in C); heavy t
//     is drawn below U just after the first light k with S_{k+1} > C_t (a
//     binary search in S) and keeps U - (S_{k+1} - C_t), aliasing heavy t + 1.
// The sweep hands each light the heavy being drawn down and moves to the next
// heavy when the current one falls below one bucket, so both forms give the
// same thresholds and aliases.
#include "alias.cuh"
#include "scan.cuh"

namespace asyrk {

namespace {

constexpr int F_BLOCK = 2048;
constexpr long long UNIT = 1LL << 32;

inline unsigned blocks_for(int64_t count) { return (unsigned)((count + 255) / 256); }

// one CTA per block of F_BLOCK rows: the block's values are staged in shared
// memory by coalesced loads, then one thread adds them in index order
__global__ void __launch_bounds__(256) k_block_sums(const double *__restrict__ v, int64_t m,
                                                    int square, double *__restrict__ part)
{
    __shared__ double sh[F_BLOCK];
    const int64_t lo = (int64_t)blockIdx.x * F_BLOCK;
    const int len = (int)(m - lo < F_BLOCK ? m - lo : F_BLOCK);
    for (int i = threadIdx.x; i < len; i += 256) {
        const double x = v[lo + i];
        sh[i] = square ? __dmul_rn(x, x) : x;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double s = 0.0;
    for (int i = 0; i < len; ++i) s = __dadd_rn(s, sh[i]);
    part[blockIdx.x] = s;
}

__global__ void k_seq_sum(const double *__restrict__ part, int64_t nb, double *__restrict__ out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int64_t b = 0; b < nb; ++b) s = __dadd_rn(s, part[b]);
    *out = s;
}

__global__ void k_differs(const double *__restrict__ w, int64_t m, unsigned *__restrict__ flag)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m && __double_as_longlong(w[i]) != __double_as_longlong(w[0])) atomicOr(flag, 1u);
}

__device__ __forceinline__ long long warp_sum_ll(long long v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ long long warp_max_ll(long long v)
{
    for (int o = 16; o > 0; o >>= 1) {
        const long long u = __shfl_down_sync(0xffffffffu, v, o);
        v = u > v ? u : v;
    }
    return v;
}

// M_i and their sum (an exact integer sum, one atomic per warp)
__global__ void k_masses(const double *__restrict__ w, int64_t m, const double *__restrict__ F,
                         long long *__restrict__ M, unsigned long long *__restrict__ sum)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    long long mi = 0;
    if (i < m) {
        const double q = __ddiv_rn(__dmul_rn(w[i], (double)m), *F);
        mi = (long long)floor(__dmul_rn(q, 4294967296.0));
        M[i] = mi;
    }
    mi = warp_sum_ll(mi);
    if ((threadIdx.x & 31) == 0 && mi) atomicAdd(sum, (unsigned long long)mi);
}

// D = m U - sum M: D >= 0 adds D / m to every row and one more to rows below D mod m
__global__ void k_mass_spread(long long *__restrict__ M, int64_t m,
                              const unsigned long long *__restrict__ sum)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const long long D = (long long)m * UNIT - (long long)*sum;
    if (i >= m || D < 0) return;
    M[i] += D / m + (i < D % m ? 1 : 0);
}

// D < 0: the overshoot comes off the first row of largest mass
__global__ void k_mass_max(const long long *__restrict__ M, int64_t m,
                           const unsigned long long *__restrict__ sum,
                           unsigned long long *__restrict__ mx)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const long long D = (long long)m * UNIT - (long long)*sum;
    if (D >= 0) return;
    long long v = i < m ? M[i] : 0;
    v = warp_max_ll(v);
    if ((threadIdx.x & 31) == 0) atomicMax(mx, (unsigned long long)v);
}

__global__ void k_mass_first_max(const long long *__restrict__ M, int64_t m,
                                 const unsigned long long *__restrict__ sum,
                                 const unsigned long long *__restrict__ mx,
                                 unsigned long long *__restrict__ first)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const long long D = (long long)m * UNIT - (long long)*sum;
    if (D >= 0 || i >= m) return;
    if ((unsigned long long)M[i] == *mx) atomicMin(first, (unsigned long long)i);
}

__global__ void k_mass_take(long long *__restrict__ M, int64_t m,
                            const unsigned long long *__restrict__ sum,
                            const unsigned long long *__restrict__ first)
{
    const long long D = (long long)m * UNIT - (long long)*sum;
    if (threadIdx.x == 0 && blockIdx.x == 0 && D < 0) M[*first] += D;
}

__global__ void k_light_flag(const long long *__restrict__ M, int64_t m, int64_t *__restrict__ flag)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) flag[i] = M[i] < UNIT ? 1 : 0;
}

// lights to [0, L), heavies to [L, m), each in index order
__global__ void k_compact(const long long *__restrict__ M, int64_t m,
                          const int64_t *__restrict__ lpos, const int64_t *__restrict__ Lp,
                          int32_t *__restrict__ idx, long long *__restrict__ de)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const long long mi = M[i];
    if (mi < UNIT) {
        const int64_t k = lpos[i];
        idx[k] = (int32_t)i;
        de[k] = UNIT - mi;
    } else {
        const int64_t k = *Lp + (i - lpos[i]);
        idx[k] = (int32_t)i;
        de[k] = mi - UNIT;
    }
}

__global__ void k_add_ll(long long *__restrict__ c, const long long *__restrict__ e, int64_t n)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) c[t] += e[t];
}

// first t in [0, n) with C[t] >= x (n if none)
__device__ __forceinline__ int64_t lower_bound_ll(const long long *C, int64_t n, long long x)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (C[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// first k in [0, n) with S[k] > x (n if none)
__device__ __forceinline__ int64_t upper_bound_ll(const long long *S, int64_t n, long long x)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (S[mid] <= x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__global__ void k_alias_lights(int64_t L, int64_t H, const long long *__restrict__ S,
                               const long long *__restrict__ C, const int32_t *__restrict__ idx,
                               const long long *__restrict__ M, RowRec *__restrict__ rec)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= L) return;
    const int64_t t = lower_bound_ll(C, H, S[k]);
    if (t >= H) return;  // no heavy left: thr = max, alias = self (set by the row pass)
    const int32_t l = idx[k];
    rec[l].thr = (unsigned)M[l];
    rec[l].alias = (unsigned)idx[L + t];
}

__global__ void k_alias_heavies(int64_t L, int64_t H, const long long *__restrict__ S,
                                const long long *__restrict__ C, const int32_t *__restrict__ idx,
                                RowRec *__restrict__ rec)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t + 1 >= H) return;  // the last heavy keeps thr = max, alias = self
    const int64_t k = upper_bound_ll(S, L + 1, C[t]);
    if (k > L) return;       // never drawn below one bucket
    const int32_t h = idx[L + t];
    rec[h].thr = (unsigned)(UNIT - (S[k] - C[t]));
    rec[h].alias = (unsigned)idx[L + t + 1];
}

struct Tmp {
    void *ptrs[16] = {};
    int n = 0;
    template <typename T>
    int alloc(T **p, size_t count)
    {
        *p = nullptr;
        cudaError_t e = cudaMalloc((void **)p, (count ? count : 1) * sizeof(T));
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            *p = nullptr;
            return set_error(e == cudaErrorMemoryAllocation ? ASYRK_ENOMEM : ASYRK_ECUDA,
                             "cudaMalloc of %zu bytes failed", count * sizeof(T));
        }
        ptrs[n++] = (void *)*p;
        return ASYRK_OK;
    }
    ~Tmp()
    {
        for (int k = 0; k < n; ++k) cudaFree(ptrs[k]);
    }
};

}  // namespace

int row_totals_and_alias(asyrk_problem *p, cudaStream_t s)
{
    const int64_t m = p->m;
    const int64_t nb = (m + F_BLOCK - 1) / F_BLOCK;
    Tmp t;
    double *part, *sums;  // sums: F, ||b||^2
    unsigned *differs;
    unsigned long long *acc;  // sum of masses, max mass, first row of max mass
    int st;
    if ((st = t.alloc(&part, (size_t)nb)) || (st = t.alloc(&sums, 2)) ||
        (st = t.alloc(&differs, 1)) || (st = t.alloc(&acc, 3)))
        return st;
    k_block_sums<<<(unsigned)nb, 256, 0, s>>>(p->w64, m, 0, part);
    k_seq_sum<<<1, 32, 0, s>>>(part, nb, sums);
    k_block_sums<<<(unsigned)nb, 256, 0, s>>>(p->b64, m, 1, part);
    k_seq_sum<<<1, 32, 0, s>>>(part, nb, sums + 1);
    ASYRK_CK(cudaMemsetAsync(differs, 0, sizeof(unsigned), s));
    k_differs<<<blocks_for(m), 256, 0, s>>>(p->w64, m, differs);
    ASYRK_CK(cudaGetLastError());
    double h_sums[2];
    unsigned h_diff = 0;
    ASYRK_CK(cudaMemcpyAsync(h_sums, sums, sizeof h_sums, cudaMemcpyDeviceToHost, s));
    ASYRK_CK(cudaMemcpyAsync(&h_diff, differs, sizeof h_diff, cudaMemcpyDeviceToHost, s));
    ASYRK_CK(cudaStreamSynchronize(s));
    if (!(h_sums[0] > 0.0) || !isfinite(h_sums[0]))
        return set_error(ASYRK_EINVAL, "||A||_F^2 is not finite");
    p->frob2 = h_sums[0];
    p->bnorm = sqrt(h_sums[1]);
    p->uniform = h_diff ? 0 : 1;
    if (p->uniform) return ASYRK_OK;

    long long *M, *de, *S, *C;
    int64_t *flag, *lpos, *scan_tmp, *Lp;
    int32_t *idx;
    if ((st = t.alloc(&M, (size_t)m)) || (st = t.alloc(&de, (size_t)m)) ||
        (st = t.alloc(&S, (size_t)m + 1)) || (st = t.alloc(&C, (size_t)m + 1)) ||
        (st = t.alloc(&flag, (size_t)m)) || (st = t.alloc(&lpos, (size_t)m)) ||
        (st = t.alloc(&scan_tmp, (size_t)scan_tmp_count(m))) || (st = t.alloc(&Lp, 1)) ||
        (st = t.alloc(&idx, (size_t)m)))
        return st;
    ASYRK_CK(cudaMemsetAsync(acc, 0, 2 * sizeof(unsigned long long), s));
    ASYRK_CK(cudaMemsetAsync(acc + 2, 0xff, sizeof(unsigned long long), s));
    const unsigned g = blocks_for(m);
    k_masses<<<g, 256, 0, s>>>(p->w64, m, sums, M, acc);
    k_mass_max<<<g, 256, 0, s>>>(M, m, acc, acc + 1);
    k_mass_first_max<<<g, 256, 0, s>>>(M, m, acc, acc + 1, acc + 2);
    k_mass_take<<<1, 32, 0, s>>>(M, m, acc, acc + 2);
    k_mass_spread<<<g, 256, 0, s>>>(M, m, acc);
    k_light_flag<<<g, 256, 0, s>>>(M, m, flag);
    ASYRK_CK(cudaGetLastError());
    if ((st = exclusive_scan(flag, lpos, m, scan_tmp, Lp, s)) != ASYRK_OK) return st;
    k_compact<<<g, 256, 0, s>>>(M, m, lpos, Lp, idx, de);
    ASYRK_CK(cudaGetLastError());
    int64_t L = 0;
    ASYRK_CK(cudaMemcpyAsync(&L, Lp, sizeof L, cudaMemcpyDeviceToHost, s));
    ASYRK_CK(cudaStreamSynchronize(s));
    const int64_t H = m - L;
    // S[0..L] (S[L] = all deficits), C[0..H) inclusive
    if ((st = exclusive_scan((const int64_t *)de, (int64_t *)S, L, scan_tmp, (int64_t *)(S + L), s)) !=
        ASYRK_OK)
        return st;
    if ((st = exclusive_scan((const int64_t *)(de + L), (int64_t *)C, H, scan_tmp,
                             (int64_t *)(C + H), s)) != ASYRK_OK)
        return st;
    if (H > 0) k_add_ll<<<blocks_for(H), 256, 0, s>>>(C, de + L, H);
    if (L > 0) k_alias_lights<<<blocks_for(L), 256, 0, s>>>(L, H, S, C, idx, M, p->rec);
    if (H > 0) k_alias_heavies<<<blocks_for(H), 256, 0, s>>>(L, H, S, C, idx, p->rec);
    ASYRK_CK(cudaGetLastError());
    ASYRK_CK(cudaStreamSynchronize(s));
    return ASYRK_OK;
}

}  // namespace asyrk
