/*
 * asyrk_oracle.c -- plain, sequential FP64 CPU restatement of randomized
 * Kaczmarz (RK) as the AsyRK paper (Liu, Wright, Sridhar, arXiv:1401.4780)
 * defines it.  TEST INFRASTRUCTURE ONLY: it is called by the tests, by the
 * smoke check and by the benchmark's CPU-baseline leg, never by the library.
 * It shares no source with the CUDA library; the two meet only through
 * seeded synthetic inputs.
 *
 * What is computed, and where the paper defines it:
 *   - problem: consistent A x = b, A is m x n, rows a_i^T, no zero rows
 *     (Section 1, "Introduction", the problem statement);
 *   - row choice: row i with probability ||a_i||^2 / ||A||_F^2 (Section 1,
 *     the description of RK just before Eq. (2));
 *   - projection: x <- x - gamma (a_i^T x - b_i) / ||a_i||^2 * a_i, which is
 *     Eq. (2) with a step-length factor gamma; gamma = 1 gives Eq. (2)
 *     exactly; the full-row update of Section 5 ("Experiments": all
 *     coordinates of supp(a_i) are updated, and on one thread the scheme is
 *     the usual RK);
 *   - the sampled row sequence: i.i.d. with replacement, as in the analysis
 *     of Section 3 (Algorithm 1).
 *
 * The paper does not say how the random row is drawn.  The draw used here
 * (and, independently, in the library) is:
 *   (u0,u1,u2,u3) = Philox4x32-10(key = (seed_lo, seed_hi),
 *                                 counter = (j_lo, j_hi, stream, 0))
 *   bucket = floor(u0 * m / 2^32);  i = (u1 < thr[bucket]) ? bucket
 *                                                         : alias[bucket]
 * with Philox4x32-10 written from Salmon, Moraes, Dror and Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3" (SC'11), and an alias table (Walker's
 * method) built as follows:
 *   - F = ||A||_F^2 is the exact sum of the w_i rounded once to the nearest
 *     double (ties to even): the w_i are added in index order into a wide
 *     fixed-point integer that loses nothing, and only the total is rounded;
 *   - integer masses M_i = floor(((w_i m) / F) 2^32) (FP64, in that order);
 *     one bucket holds U = 2^32; the D = m U - sum M_i units the floors lose
 *     go one per row from row 0 on (D/m to every row first when D >= m), and
 *     an overshoot (D < 0) comes off the first row of largest mass, so the
 *     masses add up to m U exactly;
 *   - lights (M_i < U) and heavies (M_i >= U), each list in index order;
 *   - one sweep over the lights: light l gets thr = M_l and alias = the heavy
 *     being drawn down, whose residual (initially its mass) drops by U - M_l;
 *     while that residual R is below U, the heavy gets thr = R and alias = the
 *     next heavy, whose residual becomes its mass minus (U - R); the last
 *     heavy and heavies never drawn below U keep thr = 2^32 - 1, alias =
 *     themselves (with exact masses no light is left without a heavy);
 *   - if all w_i are bit-identical, the table is skipped and i = bucket.
 * This sweep is equivalent to a form the GPU evaluates in parallel: with
 * S_k the deficit U - M of the lights before light k and C_t the excess
 * M - U of heavies 0..t, light k pairs with heavy #{t : C_t < S_k} and heavy t
 * falls below U just after the first light k with S_{k+1} > C_t.
 *
 * Shuffled sweeps (the paper's implementation visits rows without
 * replacement, reshuffled after each scan, Section 5): projection j belongs to
 * sweep k = floor(j/m) at position q = j mod m and uses row pi_k(q), where
 * pi_k is a bijection of [0, m): a 4-round balanced Feistel network on 2h bits
 * (h = max(1, ceil(log2(m)/2))) iterated until the value falls below m (cycle
 * walking; after 4096 steps, which does not happen in practice, q itself).
 * Round r maps (L, R) to (R, L xor (F(R xor K_r) and (2^h - 1))) with F
 * MurmurHash3's 32-bit finalizer (Appleby) and K_0..K_3 the four Philox words
 * at counter (k_lo, k_hi, stream, 1).
 *
 * Single-coordinate update (Algorithm 1): instead of the whole row, only the
 * entry t of supp(a_i) is updated, x_t <- x_t - gamma theta_i A_it r/||a_i||^2,
 * theta_i = ||a_i||_0, t = floor(u2 theta_i / 2^32) with u2 the third Philox
 * word of projection j (counter (j_lo, j_hi, stream, 0)).  With unit rows this
 * is Algorithm 1's step; its expectation over t is the full-row step (the
 * identity E_t[theta P_t a] = a used in the proof of Theorem 1).
 *
 * Least squares (Section 6): oracle_lsq_augment writes the square consistent
 * system [[0, phi A^T], [A, -zeta I]] (x, y) = (phi A^T b, 0) whose x-block
 * solutions are zeta x_LS; RK on it is the same projection as above.
 *
 * Arithmetic is round-to-nearest FP64 in the order written, with no FMA
 * contraction (the build passes -ffp-contract=off): w_i sums val^2 in CSR
 * order, a_i^T x sums in CSR order; F alone is exact before its one rounding.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_ENOMEM (-2)
#define OR_NOT_CONVERGED 1
#define OR_DIVERGED 2

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11): a 10-round Feistel-like        */
/* bijection of the 128-bit counter, keyed by 64 bits.                  */
/* ------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u /* golden ratio */
#define PHILOX_W1 0xBB67AE85u /* sqrt(3) - 1 */

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                          uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { /* the key schedule adds the Weyl constants */
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------ */
/* Problem checks: the paper's problem has no zero rows (Section 1).   */
/* The CSR must have row_ptr[0] = 0, non-empty rows, strictly          */
/* ascending columns in [0, n) within a row, finite values, ||a_i|| > 0 */
/* and finite b.                                                       */
/* ------------------------------------------------------------------ */
int oracle_validate(int64_t m, int64_t n, const int64_t *row_ptr,
                    const int32_t *col, const double *val, const double *b)
{
    if (m <= 0 || n <= 0 || m > 0x7fffffffLL || n > 0x7fffffffLL) return OR_EINVAL;
    if (!row_ptr || !col || !val) return OR_EINVAL;
    if (row_ptr[0] != 0) return OR_EINVAL;
    for (int64_t i = 0; i < m; ++i) {
        int64_t s = row_ptr[i], e = row_ptr[i + 1];
        if (e <= s) return OR_EINVAL; /* zero row */
        double w = 0.0;
        for (int64_t k = s; k < e; ++k) {
            if (col[k] < 0 || (int64_t)col[k] >= n) return OR_EINVAL;
            if (k > s && col[k] <= col[k - 1]) return OR_EINVAL;
            if (!isfinite(val[k])) return OR_EINVAL;
            w += val[k] * val[k];
        }
        if (!(w > 0.0) || !isfinite(w)) return OR_EINVAL;
        if (b && !isfinite(b[i])) return OR_EINVAL;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Exact sum of non-negative doubles.  Every finite double is an        */
/* integer multiple of 2^-1074 below 2^1024, so the sum of fewer than   */
/* 2^31 of them is an integer (in units of 2^-1074) of at most 2129     */
/* bits: EXACT_DIGITS base-2^32 digits, least significant first, hold   */
/* it with room to spare.  Nothing is rounded until exact_round.        */
/* ------------------------------------------------------------------ */
#define EXACT_DIGITS 68

/* digits += v, for a finite v >= 0 */
static void exact_add(uint32_t *digits, double v)
{
    if (v == 0.0) return;
    int e;
    const double f = frexp(v, &e);                  /* v = f 2^e, 1/2 <= f < 1 */
    uint64_t mant = (uint64_t)ldexp(f, 53);         /* v = mant 2^(e - 53), exactly */
    int pos = e - 53 + 1074;                        /* weight of mant's last bit, from 2^-1074 */
    while (pos < 0) { mant >>= 1; ++pos; }          /* subnormal v: the bits shifted out are 0 */
    const int q = pos / 32, r = pos % 32;
    /* the three base-2^32 digits of mant 2^r, added at digit q with carries */
    uint32_t part[3];
    part[0] = (uint32_t)(mant << r);
    part[1] = (uint32_t)(r == 0 ? mant >> 32 : mant >> (32 - r));
    part[2] = (uint32_t)(r == 0 ? 0 : mant >> (64 - r));
    uint64_t carry = 0;
    for (int k = q; k < EXACT_DIGITS; ++k) {
        const uint64_t t = (uint64_t)digits[k] + (k - q < 3 ? part[k - q] : 0) + carry;
        digits[k] = (uint32_t)t;
        carry = t >> 32;
        if (k - q >= 2 && carry == 0) break;
    }
}

/* bit b of the digit string */
static int exact_bit(const uint32_t *digits, int b)
{
    return (int)((digits[b / 32] >> (b % 32)) & 1u);
}

/* The digits' value, units of 2^-1074, rounded to the nearest double, ties to
 * even; +inf when it is 2^1024 or more after rounding. */
static double exact_round(const uint32_t *digits)
{
    int top = -1;                                   /* highest set bit */
    for (int b = 32 * EXACT_DIGITS - 1; b >= 0; --b)
        if (exact_bit(digits, b)) { top = b; break; }
    if (top < 0) return 0.0;
    if (top < 53) {                                 /* fewer than 54 bits: exact */
        uint64_t v = 0;
        for (int b = top; b >= 0; --b) v = 2 * v + (uint64_t)exact_bit(digits, b);
        return ldexp((double)v, -1074);
    }
    const int s = top - 52;                         /* the 53 kept bits are top..s */
    uint64_t mant = 0;
    for (int b = top; b >= s; --b) mant = 2 * mant + (uint64_t)exact_bit(digits, b);
    const int guard = exact_bit(digits, s - 1);
    int sticky = 0;
    for (int b = s - 2; b >= 0 && !sticky; --b) sticky = exact_bit(digits, b);
    if (guard && (sticky || (mant & 1u))) ++mant;   /* round half to even */
    return ldexp((double)mant, s - 1074);           /* mant <= 2^53: exact, or +inf */
}

/* The correctly rounded sum of n finite values v_i >= 0 (n < 2^31). */
double oracle_exact_sum(int64_t n, const double *v)
{
    uint32_t digits[EXACT_DIGITS];
    memset(digits, 0, sizeof digits);
    for (int64_t i = 0; i < n; ++i) exact_add(digits, v[i]);
    return exact_round(digits);
}

/* w_i = ||a_i||^2 in CSR order; returns F = ||A||_F^2, the exact sum of the
 * w_i rounded once. */
double oracle_row_weights(int64_t m, const int64_t *row_ptr, const double *val,
                          double *w)
{
    for (int64_t i = 0; i < m; ++i) {
        double s = 0.0;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) s += val[k] * val[k];
        w[i] = s;
    }
    return oracle_exact_sum(m, w);
}

/* The alias table (see the header): integer masses M_i = floor(q_i 2^32) with
 * q_i = (w_i m) / F, lights (M < 2^32) and heavies (M >= 2^32) each in index
 * order, and one sweep that hands each light the heavy currently being drawn
 * down; a heavy whose residual falls below 2^32 keeps that residual as its
 * threshold and hands the rest to the next heavy.  Returns 1 when all
 * weights are bit-identical (the table is then unused and left as the
 * identity), 0 otherwise, or OR_ENOMEM. */
int oracle_alias_build(int64_t m, const double *w, double F, uint32_t *thr,
                       uint32_t *alias)
{
    const int64_t U = (int64_t)1 << 32;
    int all_equal = 1;
    for (int64_t i = 1; i < m; ++i)
        if (memcmp(&w[i], &w[0], sizeof(double)) != 0) { all_equal = 0; break; }
    for (int64_t i = 0; i < m; ++i) { thr[i] = 0xffffffffu; alias[i] = (uint32_t)i; }
    if (all_equal) return 1;

    int64_t *M = (int64_t *)malloc((size_t)m * sizeof(int64_t));
    int64_t *light = (int64_t *)malloc((size_t)m * sizeof(int64_t));
    int64_t *heavy = (int64_t *)malloc((size_t)m * sizeof(int64_t));
    if (!M || !light || !heavy) { free(M); free(light); free(heavy); return OR_ENOMEM; }
    int64_t L = 0, H = 0, sum = 0;
    for (int64_t i = 0; i < m; ++i) {
        const double q = (w[i] * (double)m) / F;
        M[i] = (int64_t)floor(q * 4294967296.0);
        sum += M[i];
    }
    /* the masses must add up to m buckets: D = m U - sum units are added one
     * per row from row 0 on (D / m to every row first if D >= m), or, when the
     * rounding overshoots (D < 0), taken from the first row of largest mass */
    const int64_t D = m * U - sum;
    if (D >= 0) {
        for (int64_t i = 0; i < m; ++i) M[i] += D / m + (i < D % m ? 1 : 0);
    } else {
        int64_t a = 0;
        for (int64_t i = 1; i < m; ++i) if (M[i] > M[a]) a = i;
        M[a] += D;
    }
    for (int64_t i = 0; i < m; ++i) {
        if (M[i] < U) light[L++] = i; else heavy[H++] = i;
    }
    int64_t t = 0;                  /* the heavy being drawn down */
    int64_t R = H > 0 ? M[heavy[0]] : 0;  /* its residual mass */
    for (int64_t k = 0; k < L; ++k) {
        const int64_t l = light[k];
        if (t >= H) break;          /* no heavy left: l keeps thr = max, alias = l */
        thr[l] = (uint32_t)M[l];
        alias[l] = (uint32_t)heavy[t];
        R -= U - M[l];
        while (t < H && R < U) {    /* heavy[t] is drawn below one bucket */
            const int64_t h = heavy[t];
            if (t + 1 < H) {
                thr[h] = (uint32_t)R;
                alias[h] = (uint32_t)heavy[t + 1];
                R = M[heavy[t + 1]] - (U - R);
            }
            ++t;                    /* the last heavy keeps thr = max, alias = itself */
        }
    }
    free(M); free(light); free(heavy);
    return 0;
}

/* One draw of the row sequence at position j. */
int64_t oracle_draw_row(uint64_t seed, uint32_t stream, uint64_t j, int64_t m,
                        const uint32_t *thr, const uint32_t *alias, int uniform)
{
    uint32_t ctr[4] = {(uint32_t)j, (uint32_t)(j >> 32), stream, 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t u[4];
    oracle_philox4x32_10(ctr, key, u);
    uint32_t bucket = (uint32_t)(((uint64_t)u[0] * (uint64_t)m) >> 32);
    if (uniform) return (int64_t)bucket;
    return (u[1] < thr[bucket]) ? (int64_t)bucket : (int64_t)alias[bucket];
}

void oracle_draw_rows(uint64_t seed, uint32_t stream, uint64_t j0, int64_t count,
                      int64_t m, const uint32_t *thr, const uint32_t *alias,
                      int uniform, int32_t *rows)
{
    for (int64_t t = 0; t < count; ++t)
        rows[t] = (int32_t)oracle_draw_row(seed, stream, j0 + (uint64_t)t, m, thr,
                                           alias, uniform);
}

/* MurmurHash3's 32-bit finalizer (Appleby): an avalanche mix of 32 bits. */
static uint32_t fmix32(uint32_t h)
{
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

/* pi_k(q): position q of sweep k in the shuffled order of rows 0..m-1. */
int64_t oracle_shuffle(uint64_t seed, uint32_t stream, uint64_t k, int64_t m, int64_t q)
{
    int bits = 0;
    while (((int64_t)1 << bits) < m) ++bits;
    int h = (bits + 1) / 2;
    if (h < 1) h = 1;
    const uint64_t mask = ((uint64_t)1 << h) - 1;
    uint32_t ctr[4] = {(uint32_t)k, (uint32_t)(k >> 32), stream, 1u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t K[4];
    oracle_philox4x32_10(ctr, key, K);
    uint64_t v = (uint64_t)q;
    for (int walk = 0; walk < 4096; ++walk) {
        uint64_t L = v >> h, R = v & mask;
        for (int r = 0; r < 4; ++r) {
            uint64_t nl = R;
            uint64_t nr = L ^ ((uint64_t)fmix32((uint32_t)R ^ K[r]) & mask);
            L = nl;
            R = nr;
        }
        v = (L << h) | R;
        if ((int64_t)v < m) return (int64_t)v;
    }
    return q;
}

/* row of projection j under a sampling scheme: 0 = weighted i.i.d. (alias),
 * 1 = shuffled sweeps */
int64_t oracle_draw_row_ex(uint64_t seed, uint32_t stream, uint64_t j, int64_t m,
                           const uint32_t *thr, const uint32_t *alias, int uniform,
                           int sampling)
{
    if (sampling == 1) {
        const uint64_t k = j / (uint64_t)m;
        return oracle_shuffle(seed, stream, k, m, (int64_t)(j - k * (uint64_t)m));
    }
    return oracle_draw_row(seed, stream, j, m, thr, alias, uniform);
}

void oracle_draw_rows_ex(uint64_t seed, uint32_t stream, uint64_t j0, int64_t count, int64_t m,
                         const uint32_t *thr, const uint32_t *alias, int uniform, int sampling,
                         int32_t *rows)
{
    for (int64_t t = 0; t < count; ++t)
        rows[t] = (int32_t)oracle_draw_row_ex(seed, stream, j0 + (uint64_t)t, m, thr, alias,
                                              uniform, sampling);
}

/* ------------------------------------------------------------------ */
/* Error measures.                                                      */
/* ------------------------------------------------------------------ */
/* ||b - A x||_2 ; the paper's plotted measure is ||Ax - b|| (Section 5). */
double oracle_residual_norm(int64_t m, const int64_t *row_ptr, const int32_t *col,
                            const double *val, const double *b, const double *x,
                            double *r_out)
{
    double ss = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        double d = 0.0;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) d += val[k] * x[col[k]];
        double r = b[i] - d;
        if (r_out) r_out[i] = r;
        ss += r * r;
    }
    return sqrt(ss);
}

/* g = A^T (A x - b): the measure ||A^T(Ax-b)||^2 of Table 2. */
void oracle_normal_residual(int64_t m, int64_t n, const int64_t *row_ptr,
                            const int32_t *col, const double *val, const double *b,
                            const double *x, double *g)
{
    for (int64_t t = 0; t < n; ++t) g[t] = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        double d = 0.0;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) d += val[k] * x[col[k]];
        double r = d - b[i];
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) g[col[k]] += val[k] * r;
    }
}

static double norm2(int64_t n, const double *v)
{
    double s = 0.0;
    for (int64_t t = 0; t < n; ++t) s += v[t] * v[t];
    return sqrt(s);
}

static double err_norm(int64_t n, const double *x, const double *xs)
{
    double s = 0.0;
    for (int64_t t = 0; t < n; ++t) {
        double d = x[t] - xs[t];
        s += d * d;
    }
    return sqrt(s);
}

/* ------------------------------------------------------------------ */
/* The RK iteration, Eq. (2) with step-length gamma, steps j = j0 ..    */
/* j0+nsteps-1 of the row sequence; update 0 = the full row (Section 5),*/
/* 1 = one coordinate (Algorithm 1, see the header).  When trace arrays  */
/* are given, step t records the row, the residual r = a_i^T x - b_i    */
/* before the step and, with x_true, ||x_j - x*||^2 before the step.    */
/* w must hold ||a_i||^2 (oracle_row_weights).                          */
/* ------------------------------------------------------------------ */
void oracle_rk_steps_ex(int64_t m, const int64_t *row_ptr, const int32_t *col,
                        const double *val, const double *b, const double *w,
                        const uint32_t *thr, const uint32_t *alias, int uniform,
                        uint64_t seed, uint32_t stream, double gamma, uint64_t j0,
                        int64_t nsteps, double *x, int64_t n, const double *x_true,
                        int32_t *trace_row, double *trace_r, double *trace_err2,
                        int sampling, int update)
{
    for (int64_t t = 0; t < nsteps; ++t) {
        const uint64_t j = j0 + (uint64_t)t;
        int64_t i = oracle_draw_row_ex(seed, stream, j, m, thr, alias, uniform, sampling);
        double dot = 0.0;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) dot += val[k] * x[col[k]];
        double r = dot - b[i];
        if (trace_row) trace_row[t] = (int32_t)i;
        if (trace_r) trace_r[t] = r;
        if (trace_err2 && x_true) {
            double e = err_norm(n, x, x_true);
            trace_err2[t] = e * e;
        }
        double s = gamma * r / w[i];
        if (update == 1) {
            uint32_t ctr[4] = {(uint32_t)j, (uint32_t)(j >> 32), stream, 0u};
            uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
            uint32_t u[4];
            oracle_philox4x32_10(ctr, key, u);
            const int64_t theta = row_ptr[i + 1] - row_ptr[i];
            const int64_t pick = (int64_t)(((uint64_t)u[2] * (uint64_t)theta) >> 32);
            const int64_t k = row_ptr[i] + pick;
            x[col[k]] -= ((double)theta * s) * val[k];
        } else {
            for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) x[col[k]] -= s * val[k];
        }
    }
}

void oracle_rk_steps(int64_t m, const int64_t *row_ptr, const int32_t *col,
                     const double *val, const double *b, const double *w,
                     const uint32_t *thr, const uint32_t *alias, int uniform,
                     uint64_t seed, uint32_t stream, double gamma, uint64_t j0,
                     int64_t nsteps, double *x, int64_t n, const double *x_true,
                     int32_t *trace_row, double *trace_r, double *trace_err2)
{
    oracle_rk_steps_ex(m, row_ptr, col, val, b, w, thr, alias, uniform, seed, stream, gamma, j0,
                       nsteps, x, n, x_true, trace_row, trace_r, trace_err2, 0, 0);
}

typedef struct oracle_result {
    int64_t sweeps;      /* completed sweeps (one sweep = m steps)            */
    int64_t steps;       /* projections applied                              */
    double rel_err;      /* ||x - x*|| / ||x*|| at exit, or -1 without x*     */
    double rel_res;      /* ||b - A x|| / ||b|| at exit                       */
    int32_t status;      /* OR_OK, OR_NOT_CONVERGED, OR_DIVERGED, OR_EINVAL   */
    int32_t pad;
} oracle_result;

/* Solve to a tolerance: check every `check_every` sweeps the relative error
 * ||x - x*|| / ||x*|| when x_true is given, else ||b - Ax|| / ||b||; stop
 * when it is <= tol, or after max_sweeps sweeps (NOT_CONVERGED), or when the
 * measure is not finite or has grown by 1e30 (DIVERGED).  Steps are counted
 * from j = j0. */
int oracle_rk_solve_ex(int64_t m, int64_t n, const int64_t *row_ptr, const int32_t *col,
                       const double *val, const double *b, double *x, double gamma,
                       uint64_t seed, uint32_t stream, uint64_t j0, double tol,
                       int64_t max_sweeps, int64_t check_every, const double *x_true,
                       int sampling, int update, oracle_result *res)
{
    memset(res, 0, sizeof(*res));
    res->rel_err = -1.0;
    int st = oracle_validate(m, n, row_ptr, col, val, b);
    if (st != OR_OK || !(gamma > 0.0 && gamma < 2.0) || check_every <= 0 ||
        max_sweeps < 0) {
        res->status = OR_EINVAL;
        return OR_EINVAL;
    }
    double *w = (double *)malloc((size_t)m * sizeof(double));
    uint32_t *thr = (uint32_t *)malloc((size_t)m * sizeof(uint32_t));
    uint32_t *alias = (uint32_t *)malloc((size_t)m * sizeof(uint32_t));
    if (!w || !thr || !alias) {
        free(w); free(thr); free(alias);
        res->status = OR_ENOMEM;
        return OR_ENOMEM;
    }
    double F = oracle_row_weights(m, row_ptr, val, w);
    int uniform = oracle_alias_build(m, w, F, thr, alias);
    if (uniform < 0) {
        free(w); free(thr); free(alias);
        res->status = OR_ENOMEM;
        return OR_ENOMEM;
    }

    double ref = x_true ? norm2(n, x_true) : norm2(m, b);
    if (!(ref > 0.0)) ref = 1.0;
    double meas0 = x_true ? err_norm(n, x, x_true) / ref
                          : oracle_residual_norm(m, row_ptr, col, val, b, x, NULL) / ref;
    double meas = meas0;
    int status = OR_NOT_CONVERGED;
    uint64_t j = j0;
    int64_t sweeps = 0;
    if (meas <= tol) status = OR_OK;
    while (status == OR_NOT_CONVERGED && sweeps < max_sweeps) {
        int64_t k = check_every;
        if (k > max_sweeps - sweeps) k = max_sweeps - sweeps;
        oracle_rk_steps_ex(m, row_ptr, col, val, b, w, thr, alias, uniform, seed, stream,
                           gamma, j, k * m, x, n, NULL, NULL, NULL, NULL, sampling, update);
        j += (uint64_t)(k * m);
        sweeps += k;
        meas = x_true ? err_norm(n, x, x_true) / ref
                      : oracle_residual_norm(m, row_ptr, col, val, b, x, NULL) / ref;
        if (!isfinite(meas) || meas > 1e30 * (meas0 > 0.0 ? meas0 : 1.0)) {
            status = OR_DIVERGED;
            break;
        }
        if (meas <= tol) status = OR_OK;
    }
    res->sweeps = sweeps;
    res->steps = (int64_t)(j - j0);
    res->rel_err = x_true ? err_norm(n, x, x_true) / ref : -1.0;
    {
        double bn = norm2(m, b);
        double rn = oracle_residual_norm(m, row_ptr, col, val, b, x, NULL);
        res->rel_res = bn > 0.0 ? rn / bn : rn;
    }
    res->status = status;
    free(w); free(thr); free(alias);
    return status;
}

int oracle_rk_solve(int64_t m, int64_t n, const int64_t *row_ptr, const int32_t *col,
                    const double *val, const double *b, double *x, double gamma,
                    uint64_t seed, uint32_t stream, uint64_t j0, double tol,
                    int64_t max_sweeps, int64_t check_every, const double *x_true,
                    oracle_result *res)
{
    return oracle_rk_solve_ex(m, n, row_ptr, col, val, b, x, gamma, seed, stream, j0, tol,
                              max_sweeps, check_every, x_true, 0, 0, res);
}

/* ------------------------------------------------------------------ */
/* Section 6: least squares through a square consistent system.        */
/* ------------------------------------------------------------------ */
/* The minimiser of ||A x - b|| solves, for any zeta > 0 and phi > 0,
 *     A x - zeta y = 0,    phi A^T y = phi A^T b,
 * whose solutions have x = zeta x_LS (and y = A x_LS).  As a CSR matrix over
 * the unknowns (x, y) of length n + m the rows are, in this order:
 *   - for each column j of A with at least one nonzero (a column of zeros
 *     gives the equation 0 = 0, which is left out): the entries
 *     (n + i, phi A_ij) for i ascending, right side phi * (sum_i A_ij b_i)
 *     with the sum taken in ascending i;
 *   - for each row i of A: its entries (j, A_ij) as given, then
 *     (n + i, -zeta); right side 0.
 * The caller sizes the outputs for n + m rows and 2 nnz + m entries; the
 * return value is the number of rows written. */
int64_t oracle_lsq_augment(int64_t m, int64_t n, const int64_t *row_ptr, const int32_t *col,
                           const double *val, const double *b, double zeta, double phi,
                           int64_t *arow_ptr, int32_t *acol, double *aval, double *ab)
{
    const int64_t nnz = row_ptr[m];
    /* A^T in CSR (the CSC of A) by counting: entries of column j in row order */
    int64_t *cstart = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t *cfill = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    int64_t *trow = (int64_t *)malloc(((size_t)nnz + 1) * sizeof(int64_t));
    double *tval = (double *)malloc(((size_t)nnz + 1) * sizeof(double));
    for (int64_t k = 0; k < nnz; ++k) cstart[col[k] + 1] += 1;
    for (int64_t j = 0; j < n; ++j) cstart[j + 1] += cstart[j];
    for (int64_t j = 0; j <= n; ++j) cfill[j] = cstart[j];
    for (int64_t i = 0; i < m; ++i)
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            const int64_t p = cfill[col[k]]++;
            trow[p] = i;
            tval[p] = val[k];
        }
    int64_t r = 0, e = 0;
    arow_ptr[0] = 0;
    for (int64_t j = 0; j < n; ++j) {
        if (cstart[j + 1] == cstart[j]) continue;
        double s = 0.0;
        for (int64_t p = cstart[j]; p < cstart[j + 1]; ++p) {
            acol[e] = (int32_t)(n + trow[p]);
            aval[e] = phi * tval[p];
            ++e;
            s += tval[p] * b[trow[p]];
        }
        ab[r] = phi * s;
        arow_ptr[++r] = e;
    }
    for (int64_t i = 0; i < m; ++i) {
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            acol[e] = col[k];
            aval[e] = val[k];
            ++e;
        }
        acol[e] = (int32_t)(n + i);
        aval[e] = -zeta;
        ++e;
        ab[r] = 0.0;
        arow_ptr[++r] = e;
    }
    free(cstart); free(cfill); free(trow); free(tval);
    return r;
}
