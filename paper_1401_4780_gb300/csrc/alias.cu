// alias.cu -- ||A||_F^2, ||b||^2 and the alias table of the row weights, on the GPU.
//
// Rows are drawn with probability w_i / F (w_i = ||a_i||^2, F = ||A||_F^2,
// Section 1) through Walker's alias table.  The table is defined by one
// sequential sweep (the header of asyrk.h states it); this file evaluates the
// same table in parallel:
//   * F is the exact sum of the w_i rounded once to the nearest double (ties to
//     even).  Every finite double is an integer multiple of 2^-1074 below
//     2^1024, so the sum is an integer of at most 2129 bits in those units: each
//     thread splits its values into base-2^32 digits and adds them into 64-bit
//     digit counters (registers, then shared memory, then one global
//     accumulator per sum) with integer atomics, which are exact in any order;
//     one thread then propagates the carries and rounds.  ||b||^2 is formed the
//     same way from the b_i^2;
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
#include "devmem.cuh"
#include "scan.cuh"

namespace asyrk {

namespace {

constexpr long long UNIT = 1LL << 32;

inline unsigned blocks_for(int64_t count) { return (unsigned)((count + 255) / 256); }

// ---------------------------------------------------------------------------
// Exact sums of non-negative doubles.  Digit k of an accumulator counts units
// of 2^(32k - 1074); XDIG digits cover 2^-1074 .. 2^1102, room for the sum of
// up to 2^31 values below 2^1024.  A digit counter takes at most one 32-bit
// part per value, so it stays below 2^63 for fewer than 2^31 values.  Word
// XDIG flags a value that is not finite.
// ---------------------------------------------------------------------------
constexpr int XDIG = 68;
constexpr int XWORDS = XDIG + 1;
constexpr int XWIN = 6;  // digits a thread keeps in registers

// v = man 2^(pos - 1074) (man < 2^53); returns the digit of man's lowest bit
// and the three base-2^32 parts of man shifted to it; -1 for inf / NaN
__device__ __forceinline__ int split_exact(double v, unsigned &d0, unsigned &d1, unsigned &d2)
{
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    const int ex = (int)((bits >> 52) & 0x7ff);
    if (ex == 0x7ff) return -1;
    unsigned long long man = bits & ((1ULL << 52) - 1);
    int pos = 0;  // subnormal (or zero): man 2^-1074
    if (ex != 0) {
        man |= 1ULL << 52;
        pos = ex - 1;
    }
    const int r = pos & 31;
    d0 = (unsigned)(man << r);
    d1 = (unsigned)(r ? man >> (32 - r) : man >> 32);
    d2 = r ? (unsigned)(man >> (64 - r)) : 0u;
    return pos >> 5;
}

// acc[0..XWORDS) += the digits of v[i] (squared when square) for i < n; one
// CTA's counters are gathered in shared memory before the global atomics.
__global__ void __launch_bounds__(256) k_exact_accumulate(const double *__restrict__ v, int64_t n,
                                                          int square,
                                                          unsigned long long *__restrict__ acc)
{
    __shared__ unsigned long long sh[XWORDS];
    for (int k = threadIdx.x; k < XWORDS; k += blockDim.x) sh[k] = 0;
    __syncthreads();
    // a window of XWIN digits in registers, placed at the thread's first value
    unsigned long long win[XWIN];
#pragma unroll
    for (int k = 0; k < XWIN; ++k) win[k] = 0;
    int base = -1;
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double x = v[i];
        if (square) x = __dmul_rn(x, x);
        unsigned d0, d1, d2;
        const int q = split_exact(x, d0, d1, d2);
        if (q < 0) {
            bad = true;
            continue;
        }
        if (base < 0) base = min(max(q - 1, 0), XDIG - XWIN);
        const int o = q - base;
        if (o >= 0 && o + 2 < XWIN) {
#pragma unroll
            for (int k = 0; k < XWIN; ++k)
                win[k] += k == o ? d0 : k == o + 1 ? d1 : k == o + 2 ? d2 : 0u;
        } else {
            atomicAdd(&sh[q], (unsigned long long)d0);
            atomicAdd(&sh[q + 1], (unsigned long long)d1);
            atomicAdd(&sh[q + 2], (unsigned long long)d2);
        }
    }
    if (base >= 0) {
#pragma unroll
        for (int k = 0; k < XWIN; ++k)
            if (win[k]) atomicAdd(&sh[base + k], win[k]);
    }
    if (bad) atomicOr(&sh[XDIG], 1ULL);
    __syncthreads();
    for (int k = threadIdx.x; k < XWORDS; k += blockDim.x)
        if (sh[k]) atomicAdd(&acc[k], sh[k]);
}

// out[s] = accumulator s rounded to the nearest double, ties to even (inf
// from 2^1024 on, NaN when a value was not finite); one thread per sum
__global__ void k_exact_round(const unsigned long long *__restrict__ acc, int count,
                              double *__restrict__ out)
{
    const int s = threadIdx.x;
    if (s >= count) return;
    const unsigned long long *a = acc + (size_t)s * XWORDS;
    if (a[XDIG]) {
        out[s] = __longlong_as_double(0x7ff8000000000000LL);
        return;
    }
    unsigned dig[XDIG];
    unsigned long long carry = 0;
    for (int k = 0; k < XDIG; ++k) {
        const unsigned long long t = a[k] + carry;  // a[k] < 2^63, carry < 2^32
        dig[k] = (unsigned)t;
        carry = t >> 32;
    }
    int top = XDIG - 1;
    while (top >= 0 && dig[top] == 0) --top;
    if (top < 0) {
        out[s] = 0.0;
        return;
    }
    const int nbits = 32 * top + 32 - __clz(dig[top]);  // bit length of the sum
    if (nbits <= 53) {
        // below 2^53 units of 2^-1074: the bit pattern of the double is the
        // integer itself (subnormal below 2^52, exponent field 1 above)
        const unsigned long long V =
            (unsigned long long)dig[0] | (top >= 1 ? (unsigned long long)dig[1] << 32 : 0ULL);
        out[s] = __longlong_as_double((long long)V);
        return;
    }
    const int sh = nbits - 53;  // bits [sh, nbits) are kept
    // the 53 kept bits, the guard bit below them and whether anything lower is set
    auto bit = [&](int b) -> unsigned { return (dig[b >> 5] >> (b & 31)) & 1u; };
    unsigned long long man = 0;
    for (int b = nbits - 1; b >= sh; --b) man = (man << 1) | bit(b);
    const unsigned guard = bit(sh - 1);
    bool sticky = false;
    for (int k = 0; k < ((sh - 1) >> 5) && !sticky; ++k) sticky = dig[k] != 0;
    if (!sticky && ((sh - 1) & 31)) sticky = (dig[(sh - 1) >> 5] & ((1u << ((sh - 1) & 31)) - 1u)) != 0;
    if (guard && (sticky || (man & 1ULL))) ++man;
    int e = sh + 1;  // biased exponent of man 2^(sh - 1074), man in [2^52, 2^53)
    if (man >> 53) {
        man >>= 1;
        ++e;
    }
    if (e >= 0x7ff) {
        out[s] = __longlong_as_double(0x7ff0000000000000LL);
        return;
    }
    out[s] = __longlong_as_double((long long)(((unsigned long long)e << 52) | (man & ((1ULL << 52) - 1))));
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

// temporaries from the problems' pool, ordered on the set-up stream and
// handed back on it when the set-up ends
struct Tmp {
    cudaStream_t s;
    void *ptrs[16] = {};
    int n = 0;
    explicit Tmp(cudaStream_t stream) : s(stream) {}
    template <typename T>
    int alloc(T **p, size_t count)
    {
        const int st = devmem_alloc_n(p, count, s);
        if (st != ASYRK_OK) return st;
        ptrs[n++] = (void *)*p;
        return ASYRK_OK;
    }
    ~Tmp()
    {
        for (int k = 0; k < n; ++k) devmem_free(ptrs[k], s);
    }
};

}  // namespace

int row_totals_and_alias(asyrk_problem *p, cudaStream_t s)
{
    const int64_t m = p->m;
    Tmp t(s);
    double *sums;  // sums: F, ||b||^2
    unsigned *differs;
    unsigned long long *acc;    // sum of masses, max mass, first row of max mass
    unsigned long long *exact;  // the two exact accumulators
    int st;
    if ((st = t.alloc(&sums, 2)) || (st = t.alloc(&differs, 1)) || (st = t.alloc(&acc, 3)) ||
        (st = t.alloc(&exact, 2 * XWORDS)))
        return st;
    // enough CTAs to fill the GPU; each thread sweeps its share in registers
    const int64_t want = (m + 255) / 256;
    const unsigned gx = (unsigned)(want < 4LL * p->sm_count ? want : 4LL * p->sm_count);
    ASYRK_CK(cudaMemsetAsync(exact, 0, 2 * XWORDS * sizeof(unsigned long long), s));
    k_exact_accumulate<<<gx, 256, 0, s>>>(p->w64, m, 0, exact);
    k_exact_accumulate<<<gx, 256, 0, s>>>(p->b64, m, 1, exact + XWORDS);
    k_exact_round<<<1, 32, 0, s>>>(exact, 2, sums);
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
    if (!isfinite(h_sums[1])) return set_error(ASYRK_EINVAL, "||b||^2 is not finite");
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
