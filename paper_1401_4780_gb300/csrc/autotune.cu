// autotune.cu -- asyrk_autotune: choose the projection kernel's launch shape by
// timing it on the problem itself.
//
// The shape is the sub-warp width G (1..32 lanes per row, hence 32/G rows per warp)
// and the number of concurrent workers W.  W never exceeds the Cor. 2
// estimate of how many workers keep the rate near the sequential one; within
// that, the fastest measured shape wins.  Results are kept per (value dtype,
// row-length class, SM count) so that problems of the same kind reuse them.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>
#include <tuple>

#include "batch.cuh"

namespace asyrk {

struct TuneVal {
    int G;
    double frac;  // workers as a fraction of the resident maximum
    double rate;
};

using TuneKey = std::tuple<int, long long, int>;  // dtype, row-length class, SM count

static std::mutex g_tune_mu;
static std::map<TuneKey, TuneVal> g_tune;
static bool g_tune_loaded = false;

static long long len_class(int64_t max_len)
{
    long long c = 1;
    while (c < max_len) c <<= 1;
    return c;
}

static void load_locked()
{
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = getenv("ASYRK_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    int dt, sms, G;
    long long lc;
    double frac, rate;
    while (fscanf(f, "%d %lld %d %d %lf %lf", &dt, &lc, &sms, &G, &frac, &rate) == 6)
        if (G >= 1 && G <= 32 && (G & (G - 1)) == 0 && frac > 0.0 && frac <= 1.0)
            g_tune[TuneKey(dt, lc, sms)] = TuneVal{G, frac, rate};
    fclose(f);
}

static void save_locked()
{
    const char *path = getenv("ASYRK_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = fopen(path, "w");
    if (!f) return;
    for (const auto &kv : g_tune)
        fprintf(f, "%d %lld %d %d %.6f %.6e\n", std::get<0>(kv.first), std::get<1>(kv.first),
                std::get<2>(kv.first), kv.second.G, kv.second.frac, kv.second.rate);
    fclose(f);
}

static int current_sms()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return sms;
}

// tuned (G, fraction of resident workers) for this kind of problem, if any
bool tuned_shape(int dtype, int64_t max_len, int *G, double *frac)
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    load_locked();
    auto it = g_tune.find(TuneKey(dtype, len_class(max_len), current_sms()));
    if (it == g_tune.end()) return false;
    *G = it->second.G;
    *frac = it->second.frac;
    return true;
}

int tuned_subwarp(int dtype, int64_t max_len, int64_t nnz, int64_t m, bool *found)
{
    (void)nnz;
    (void)m;
    int G = 0;
    double frac = 1.0;
    *found = tuned_shape(dtype, max_len, &G, &frac);
    return *found ? G : 0;
}

}  // namespace asyrk

using namespace asyrk;

extern "C" int asyrk_autotune(asyrk_problem *p, int64_t trial, int force, asyrk_tune_result *res)
{
    if (!p || !res || trial < 0) return set_error(ASYRK_EINVAL, "bad autotune arguments");
    memset(res, 0, sizeof *res);
    const bool x_f64 = p->dtype == ASYRK_F64;
    const long long cap = tau_cap_estimate(p->m, p->n);
    int G = 0;
    double frac = 1.0;
    if (!force && tuned_shape(p->dtype, p->max_len, &G, &frac)) {
        int maxw = 0;
        int st = project_max_workers(p, x_f64, G, &maxw);
        if (st != ASYRK_OK) return st;
        long long W = (long long)(frac * maxw);
        if (W > cap) W = cap;
        res->subwarp = G;
        res->workers = (int)(W < 1 ? 1 : W);
        res->from_cache = 1;
        std::lock_guard<std::mutex> lock(g_tune_mu);
        res->projections_per_s = g_tune[TuneKey(p->dtype, len_class(p->max_len), p->sm_count)].rate;
        return ASYRK_OK;
    }
    int st = ensure_workspace(p);
    if (st != ASYRK_OK) return st;
    if (!x_f64 && p->rec_b_is_residual && (st = launch_restore_rec_b(p, 0)) != ASYRK_OK) return st;
    if (trial == 0) trial = 2 * p->m < (1LL << 22) ? 2 * p->m : (1LL << 22);
    cudaEvent_t e0 = p->ev[0], e1 = p->ev[1];
    double best = -1.0;
    int bestG = 0, bestW = 0;
    double bestFrac = 1.0;
    const double fracs[3] = {0.5, 0.75, 1.0};
    for (int g = 1; g <= 32; g *= 2) {
        // rows must fit the registers (two 4G-entry chunks) unless g is the widest
        if (8LL * g < p->max_len && g < 32) continue;
        // and should not leave most lanes idle
        if (4LL * g >= 2 * (p->max_len > 4 ? p->max_len : 4) && g > 2) continue;
        int maxw = 0;
        if ((st = project_max_workers(p, x_f64, g, &maxw)) != ASYRK_OK) return st;
        long long prevW = -1;
        for (double fr : fracs) {
            long long W = (long long)(fr * maxw);
            if (W > cap) W = cap;
            if (W < 1) W = 1;
            if (W == prevW) continue;
            prevW = W;
            float ms_best = 1e30f;
            for (int rep = 0; rep < 2; ++rep) {
                ASYRK_CK(cudaMemset(p->xw, 0, p->n * (x_f64 ? 8 : 4)));
                ProjectLaunch L;
                L.p = p;
                L.x = p->xw;
                L.x_f64 = x_f64;
                L.gamma = 1.0;
                L.j0 = 0x4000000000000000ULL + (unsigned long long)rep * (unsigned long long)trial;
                L.count = (unsigned long long)trial;
                L.stream_id = 0x7475u;  // a Philox stream no solve uses
                L.workers = (int)W;
                L.subwarp = g;
                L.sequential = false;
                L.exclusive = true;
                L.b_from_rec = !x_f64;
                L.stream = 0;
                ASYRK_CK(cudaEventRecord(e0, 0));
                if ((st = launch_project(L)) != ASYRK_OK) return st;
                ASYRK_CK(cudaEventRecord(e1, 0));
                ASYRK_CK(cudaEventSynchronize(e1));
                float ms = 0.f;
                ASYRK_CK(cudaEventElapsedTime(&ms, e0, e1));
                if (ms < ms_best) ms_best = ms;
            }
            res->trials += 1;
            const double rate = (double)trial / (ms_best / 1e3);
            if (rate > best) {
                best = rate;
                bestG = g;
                bestW = (int)W;
                bestFrac = (double)W / (double)maxw;
            }
        }
    }
    if (bestG == 0) return set_error(ASYRK_EINVAL, "no launch shape fits this problem");
    res->subwarp = bestG;
    res->workers = bestW;
    res->projections_per_s = best;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        load_locked();
        g_tune[TuneKey(p->dtype, len_class(p->max_len), p->sm_count)] =
            TuneVal{bestG, bestFrac > 1.0 ? 1.0 : bestFrac, best};
        save_locked();
    }
    return ASYRK_OK;
}
