/*
 * cpu_baseline_mt.c -- the paper's own multicore scheme (Section 5) on the host
 * cores, as a CPU baseline for the benchmark.  BENCHMARK INFRASTRUCTURE ONLY:
 * it is not a parity oracle (threads race by design, so runs are not
 * reproducible) and the CUDA library never calls it.
 *
 * What it runs (Section 5, "Experiments"): T threads share x; thread t owns the
 * contiguous slice of rows [m t / T, m (t+1) / T) and scans it in a random
 * order, reshuffled (Fisher-Yates) after every scan; for each row it reads x on
 * supp(a_i) without locks, forms r = a_i^T x - b_i and applies
 * x_k -= gamma r a_ik / ||a_i||^2 to every k in supp(a_i) with an atomic add
 * (a compare-and-swap loop on the 32-bit pattern).  Values, b and x are FP32,
 * as in the GPU's FP32 path.  The shuffles use splitmix64 (Steele, Lea, Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014), one stream
 * per thread.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

typedef struct {
    const int64_t *row_ptr;
    const int32_t *col;
    const float *val;
    const float *b;
    const float *inv_w;
    float *x;
    float gamma;
    int64_t lo, hi;
    int64_t scans;
    uint64_t rng;
    int64_t done;
} slice_t;

static uint64_t splitmix64(uint64_t *s)
{
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static float load_f32(const float *p)
{
    uint32_t u = __atomic_load_n((const uint32_t *)p, __ATOMIC_RELAXED);
    float f;
    memcpy(&f, &u, 4);
    return f;
}

static void add_f32(float *p, float v)
{
    uint32_t old = __atomic_load_n((uint32_t *)p, __ATOMIC_RELAXED), nw;
    do {
        float f;
        memcpy(&f, &old, 4);
        f += v;
        memcpy(&nw, &f, 4);
    } while (!__atomic_compare_exchange_n((uint32_t *)p, &old, nw, 1, __ATOMIC_RELAXED,
                                          __ATOMIC_RELAXED));
}

static void *worker(void *arg)
{
    slice_t *s = (slice_t *)arg;
    const int64_t len = s->hi - s->lo;
    if (len <= 0) return NULL;
    int64_t *order = (int64_t *)malloc((size_t)len * sizeof(int64_t));
    if (!order) return NULL;
    for (int64_t q = 0; q < len; ++q) order[q] = s->lo + q;
    for (int64_t scan = 0; scan < s->scans; ++scan) {
        for (int64_t q = len - 1; q > 0; --q) {
            const int64_t r = (int64_t)(splitmix64(&s->rng) % (uint64_t)(q + 1));
            const int64_t t = order[q];
            order[q] = order[r];
            order[r] = t;
        }
        for (int64_t q = 0; q < len; ++q) {
            const int64_t i = order[q];
            float d = 0.0f;
            for (int64_t k = s->row_ptr[i]; k < s->row_ptr[i + 1]; ++k)
                d += s->val[k] * load_f32(s->x + s->col[k]);
            const float c = -s->gamma * (d - s->b[i]) * s->inv_w[i];
            for (int64_t k = s->row_ptr[i]; k < s->row_ptr[i + 1]; ++k)
                add_f32(s->x + s->col[k], c * s->val[k]);
        }
        s->done += len;
    }
    free(order);
    return NULL;
}

/* Runs `scans` scans of every thread's slice from the given x (updated in
 * place); returns the projections done and writes the wall time in seconds.
 * inv_w[i] = 1/||a_i||^2.  Returns -1 if a thread could not be started. */
int64_t cpu_asyrk_mt(int64_t m, const int64_t *row_ptr, const int32_t *col, const float *val,
                     const float *b, const float *inv_w, float *x, float gamma, int threads,
                     int64_t scans, uint64_t seed, double *seconds)
{
    if (threads < 1) threads = 1;
    slice_t *sl = (slice_t *)calloc((size_t)threads, sizeof(slice_t));
    pthread_t *th = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
    if (!sl || !th) {
        free(sl);
        free(th);
        return -1;
    }
    for (int t = 0; t < threads; ++t) {
        sl[t] = (slice_t){row_ptr, col, val, b, inv_w, x, gamma, m * t / threads,
                          m * (t + 1) / threads, scans, seed ^ (0xA5A5ull * (uint64_t)(t + 1)), 0};
    }
    struct timespec t0, t1;
    clock_gettime(CLOCK_MONOTONIC, &t0);
    int started = 0;
    for (; started < threads; ++started)
        if (pthread_create(&th[started], NULL, worker, &sl[started]) != 0) break;
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    clock_gettime(CLOCK_MONOTONIC, &t1);
    int64_t done = 0;
    for (int t = 0; t < started; ++t) done += sl[t].done;
    if (seconds) *seconds = (double)(t1.tv_sec - t0.tv_sec) + 1e-9 * (double)(t1.tv_nsec - t0.tv_nsec);
    free(sl);
    free(th);
    return started == threads ? done : -1;
}
