// w1_tune.cu -- autotuner for the level kernels.
//
// For one level (nx x ny, norm) and a batch of B pairs that advance together,
// every configuration that can run the level is timed on a synthetic problem
// with CUDA events:
//   * on chip (path 1) with each feasible cluster size (bands of whole rows,
//     at most 4096 nodes per CTA, or 16384 with the wide layout);
//   * streaming, one step per launch (path 2);
//   * streaming with temporal blocking (path 3, nx % 4 == 0), each tile shape
//     and depth of the kernel's table.
// The measured quantity is the time of one step of the whole batch, so the
// choice accounts for how many pairs fit on the GPU at once (a configuration
// with fewer CTAs per pair is slower for one pair but may finish a large batch
// sooner).  Objective 1 tunes for one pair alone (latency), objective 2 for the
// given batch (throughput).  Results are cached per (device, nx, ny, norm,
// batch) for the process and, if W1_AUTOTUNE_CACHE names a file, across
// processes (one line per entry).
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "w1_internal.h"

using namespace w1;

namespace {

struct TuneKey {
    int dev, nx, ny, norm, batch;
    bool operator<(const TuneKey& o) const
    {
        return std::tie(dev, nx, ny, norm, batch) < std::tie(o.dev, o.nx, o.ny, o.norm, o.batch);
    }
};

std::mutex g_tune_mu;
std::map<TuneKey, w1_level_choice> g_tune_cache;
bool g_tune_loaded = false;
thread_local std::string g_tune_err;

const char* cache_path() { return std::getenv("W1_AUTOTUNE_CACHE"); }

void load_cache_file()
{
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char* p = cache_path();
    if (!p) return;
    FILE* f = std::fopen(p, "r");
    if (!f) return;
    TuneKey k;
    w1_level_choice c;
    while (std::fscanf(f, "%d %d %d %d %d %d %d %d %lf %d %d", &k.dev, &k.nx, &k.ny, &k.norm, &k.batch, &c.path,
                       &c.cluster, &c.batch, &c.us_per_step, &c.concurrent, &c.tile) == 11)
        g_tune_cache[k] = c;
    std::fclose(f);
}

void append_cache_file(const TuneKey& k, const w1_level_choice& c)
{
    const char* p = cache_path();
    if (!p) return;
    FILE* f = std::fopen(p, "a");
    if (!f) return;
    std::fprintf(f, "%d %d %d %d %d %d %d %d %.6f %d %d\n", k.dev, k.nx, k.ny, k.norm, k.batch, c.path, c.cluster,
                 c.batch, c.us_per_step, c.concurrent, c.tile);
    std::fclose(f);
}

// Times `steps` steps of one candidate on `pairs` pairs; microseconds per step
// of the whole batch (< 0 on failure).
double time_candidate(int norm, int path, int cluster, int tile, int nx, int ny, int pairs, int steps, float* buf,
                      double* part, Ctl* ctl, cudaStream_t s)
{
    const size_t n = (size_t)nx * ny, plane = n * pairs;
    float* rho = buf;
    float* A[3] = {buf + plane, buf + 2 * plane, buf + 3 * plane};
    float* B[3] = {buf + 4 * plane, buf + 5 * plane, buf + 6 * plane};
    const double h = 1.0 / (nx > ny ? nx : ny);
    IterArgs it{};
    it.nx = nx;
    it.ny = ny;
    it.mu = (float)(0.5 * h / (2.0 * 1.4142135623730951));
    it.tau = it.mu;
    it.ih = (float)(1.0 / h);
    it.h = h;
    it.tol = 0.0;
    it.K = 32;
    it.fixed = 1;
    it.budget_ns = 10ull * 1000000000ull;
    it.stride = (long long)n;
    it.ctl = nullptr;
    auto run = [&](int nsteps) -> cudaError_t {
        if (path == 1) {
            ResArgs a{};
            a.m1 = A[0];
            a.m2 = A[1];
            a.phi = A[2];
            a.rho = rho;
            a.pairs = pairs;
            a.it = it;
            a.it.cap = nsteps;
            return launch_resident(norm, cluster, a, s);
        }
        const int per = path == 3 ? tblock_depth(tile) : 1;
        const int launches = nsteps / per;
        for (int k = 0; k < launches; ++k) {
            StepArgs a{};
            float** src = (k & 1) ? B : A;
            float** dst = (k & 1) ? A : B;
            a.m1 = src[0];
            a.m2 = src[1];
            a.phi = src[2];
            a.rho = rho;
            a.m1o = dst[0];
            a.m2o = dst[1];
            a.phio = dst[2];
            a.rows = stream_rows_auto(nx, ny, pairs);
            a.pairs = pairs;
            a.it = it;
            a.it.ctl = ctl;
            a.part = part;
            a.use_cond = 0;
            a.tile = tile;
            cudaError_t e = path == 3 ? launch_tblock(norm, false, a, s) : launch_step(norm, false, a, s);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    };
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return -1.0;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return -1.0;
    }
    double us = -1.0;
    if (run(32) == cudaSuccess && cudaEventRecord(e0, s) == cudaSuccess && run(steps) == cudaSuccess &&
        cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) us = ms * 1e3 / steps;
    }
    cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return us;
}

}  // namespace

extern "C" w1_status w1_autotune_level(int nx, int ny, int norm, int batch, int objective, int steps,
                                       w1_level_choice* best, w1_level_choice* all, int* n_all)
{
    NvtxRange range("w1 autotune %dx%d p%d", nx, ny, norm);
    if (nx < 1 || ny < 1 || batch < 1 || !best || objective < 1 || objective > 3) {
        g_tune_err = "bad arguments to w1_autotune_level";
        return W1_ERR_INVALID_ARG;
    }
    if (norm != W1_NORM_L1 && norm != W1_NORM_L2 && norm != W1_NORM_LINF) {
        g_tune_err = "norm must be 1, 2 or 3";
        return W1_ERR_INVALID_ARG;
    }
    if (steps < 32) steps = 32;
    steps = (steps + 31) / 32 * 32;
    const int B = objective == 2 ? batch : 1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        g_tune_err = "cudaGetDevice failed";
        return W1_ERR_CUDA;
    }
    const TuneKey key{dev, nx, ny, norm, objective == 3 ? -1 : B};  // -1: the SM-time objective
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        load_cache_file();
        auto itc = g_tune_cache.find(key);
        if (itc != g_tune_cache.end() && !all) {
            *best = itc->second;
            if (n_all) *n_all = 0;
            return W1_OK;
        }
    }
    if (resident_prepare(dev) != cudaSuccess) {
        cudaGetLastError();
        g_tune_err = "kernel attributes could not be set";
        return W1_ERR_CUDA;
    }
    // the pairs timed together: the batch, or as many as 2 GiB of state allow
    // (the time is then scaled to the batch)
    const size_t n = (size_t)nx * ny;
    const size_t per_pair = 7 * n * sizeof(float);
    int P = B;
    if ((size_t)P * per_pair > (2ull << 30)) P = (int)((2ull << 30) / per_pair) > 0 ? (int)((2ull << 30) / per_pair) : 1;
    std::vector<w1_level_choice> cands;
    const int cs[5] = {1, 2, 4, 8, 16};
    for (int c : cs)
        if (resident_fits(nx, ny, c) && resident_cluster_ok(norm, c, nx, ny) > 0)
            cands.push_back(w1_level_choice{1, c, B, 0.0, resident_cluster_ok(norm, c, nx, ny), 0});
    cands.push_back(w1_level_choice{2, 0, B, 0.0, 1, 0});
    if (nx % 4 == 0)
        for (int tile = 0; tile < W1_TILE_VARIANTS; ++tile) cands.push_back(w1_level_choice{3, 0, B, 0.0, 1, tile});

    float* buf = nullptr;
    double* part = nullptr;
    Ctl* ctl = nullptr;
    cudaStream_t s = nullptr;
    size_t pd = step_part_doubles(nx, ny, stream_rows_auto(nx, ny, P), P);
    if (tblock_part_doubles(nx, ny, P) > pd) pd = tblock_part_doubles(nx, ny, P);
    cudaError_t e = cudaMalloc(&buf, (size_t)P * per_pair);
    if (e == cudaSuccess) e = cudaMalloc(&part, pd * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&ctl, (size_t)P * sizeof(Ctl));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, (size_t)P * per_pair, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctl, 0, (size_t)P * sizeof(Ctl), s);
    if (e == cudaSuccess) {
        // a zero-mean density per pair: +1 on the first half of the nodes, -1 on the second
        std::vector<float> r(n);
        for (size_t k = 0; k < n; ++k) r[k] = (k < n / 2) ? 1.f : -1.f;
        if (n % 2) r[n - 1] = 0.f;
        for (int q = 0; q < P && e == cudaSuccess; ++q)
            e = cudaMemcpyAsync(buf + (size_t)q * n, r.data(), n * sizeof(float), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    w1_status ret = W1_OK;
    int n_ok = 0;
    w1_level_choice pick{0, 0, B, 0.0, 0, 0};
    double best_cost = 1e300;
    if (e != cudaSuccess) {
        g_tune_err = std::string("autotune allocation: ") + cudaGetErrorString(e);
        ret = W1_ERR_CUDA;
    } else {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 152;
        for (auto& c : cands) {
            const double us = time_candidate(norm, c.path, c.cluster, c.tile, nx, ny, P, steps, buf, part, ctl, s);
            if (us <= 0.0) continue;
            c.us_per_step = us * (double)B / (double)P;
            // objective 3: SM-time of a step (on-chip levels hold one CTA per SM; a
            // streaming launch spreads over the whole GPU)
            const double cost = objective == 3 ? c.us_per_step * (c.path == 1 ? c.cluster : sms) : c.us_per_step;
            if (cost < best_cost) {
                best_cost = cost;
                pick = c;
            }
            if (all && n_ok < W1_TUNE_MAX_CANDIDATES) all[n_ok] = c;
            ++n_ok;
        }
        if (n_ok == 0) {
            g_tune_err = "no configuration could run this level";
            ret = W1_ERR_UNSUPPORTED;
        }
    }
    cudaFree(buf);
    cudaFree(part);
    cudaFree(ctl);
    if (s) cudaStreamDestroy(s);
    cudaGetLastError();
    if (n_all) *n_all = n_ok < W1_TUNE_MAX_CANDIDATES ? n_ok : W1_TUNE_MAX_CANDIDATES;
    if (ret != W1_OK) return ret;
    *best = pick;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (!g_tune_cache.count(key)) {
        g_tune_cache[key] = pick;
        append_cache_file(key, pick);
    }
    return W1_OK;
}

extern "C" const char* w1_autotune_last_error(void) { return g_tune_err.c_str(); }
