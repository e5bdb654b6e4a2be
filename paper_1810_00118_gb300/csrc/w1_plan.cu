// w1_plan.cu -- host driver and C ABI of the GB300 multilevel W1 solver.
//
// A plan fixes the grid, the level hierarchy of Algorithm 3 (h_l = 2^{L-l} h,
// Sec. 3.2), the norm, the tolerances and the batch size B, and owns one device
// arena:
//   per-pair control blocks | partial sums | FP64 scratch for the certificate |
//   per level: rho_l, state A (m1, m2, phi), state B (streaming levels only),
// each plane holding B pairs back to back.  The level sequence (restriction,
// level starts, level solves) is captured once into a CUDA graph.  Resident
// levels are single launches (one CTA or cluster per pair) that run every pair
// to its stop test on the device; streaming levels are conditional WHILE nodes
// whose body is K batched steps, the last of which forms each pair's R^k,
// retires converged pairs, and lets a one-block kernel set the condition while
// any pair is still active.  A solve is: prep (rho = rho0 - rho1, mass check)
// -> graph -> final statistics -> one device-to-host copy of the control
// blocks.  No host synchronisation happens between the first and the last.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "w1_internal.h"

using namespace w1;

namespace {

thread_local std::string g_err;

w1_status fail(w1_status s, const std::string& msg)
{
    g_err = msg;
    return s;
}

#define W1_CK(call)                                                                                \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) {                                                                   \
            cudaGetLastError();                                                                    \
            return fail(e_ == cudaErrorMemoryAllocation ? W1_ERR_NOMEM : W1_ERR_CUDA,              \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                       \
        }                                                                                          \
    } while (0)

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

std::mutex g_prep_mu;
bool g_prepared[64] = {};

w1_status prepare_device(int dev)
{
    std::lock_guard<std::mutex> lk(g_prep_mu);
    if (dev >= 0 && dev < 64 && g_prepared[dev]) return W1_OK;
    W1_CK(resident_prepare(dev));
    if (dev >= 0 && dev < 64) g_prepared[dev] = true;
    return W1_OK;
}

// Per-device constant tables of the prox-PDHG path (twiddles), made once.
std::mutex g_pd_mu;
float2* g_pd_tw[64] = {};

w1_status pd_device_tables(int dev, const float2** tw)
{
    std::lock_guard<std::mutex> lk(g_pd_mu);
    if (dev < 0 || dev >= 64) return fail(W1_ERR_CUDA, "device index out of range");
    if (!g_pd_tw[dev]) {
        std::vector<float2> h(pd_twiddle_count());
        pd_twiddles(h.data());
        float2* d = nullptr;
        W1_CK(cudaMalloc(&d, h.size() * sizeof(float2)));
        cudaError_t e = cudaMemcpy(d, h.data(), h.size() * sizeof(float2), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(d);
            cudaGetLastError();
            return fail(W1_ERR_CUDA, std::string("twiddle table: ") + cudaGetErrorString(e));
        }
        W1_CK(pd_prepare());
        g_pd_tw[dev] = d;
    }
    *tw = g_pd_tw[dev];
    return W1_OK;
}

}  // namespace

struct LevelPlan {
    int nx, ny;
    double h;
    float mu, tau;
    double tol;
    int path;     // 1 resident, 2 streaming
    int cluster;  // resident cluster size
    int rows;     // streaming march length
    int tile;     // path 3: tile variant (w1_options.tile)
    float* rho;
    float* m1[2];
    float* m2[2];
    float* phi[2];
    // prox-PDHG levels (path 4): phi (vector), phibar, Poisson residual and
    // transpose scratch, eigenvalue tables
    float* pd[6];
    float* lam;  // nx + ny entries
};

struct w1_plan {
    int device;
    int nx, ny, L, norm, batch;
    double h, tol;
    w1_options opt;
    LevelPlan lv[W1_MAX_LEVELS];
    size_t ws_bytes;
    char* ws;
    bool own_ws;
    Ctl* ctl;
    double* part;
    size_t part_doubles;
    double* q;
    Ctl* host_ctl;
    cudaStream_t cap_stream;
    cudaStream_t body_stream;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    bool graph_ok;
    float* in0;
    float* in1;
    float* flux_d;
    cudaEvent_t host_done;  // host-buffer solves wait on it asleep (blocking sync)
    int last_batch;
    const float2* tw;  // prox-PDHG twiddle table (per device)
};

namespace w1 {
int fault_halo_rank()
{
    const char* e = std::getenv("W1_FAULT_HALO_RANK");
    if (!e || !*e) return 0;
    const int r = std::atoi(e);
    return r >= 0 && r < 16 ? r + 1 : 0;
}
}  // namespace w1

// The calibrated schedules (w1_options.schedule = 1), p = 1 then p = 2: the
// scale of eq. stop_tol's eps_L, the alpha of eq. tol_formula_propose and the
// step-size factor theta and the step ratio tau / mu.  Measured on the 512^2
// ellipse-texture pairs against their converged W1 (saddle-value estimate),
// over eps_L scales, alpha in {-1, 0, 1/2}, theta in {1/2, 1} and tau / mu from
// 0.005 to 4: the fastest whose worst relative error over the calibration pairs
// was at most 2.5e-5, a factor of four below 1e-4.  theta = 1 is the footnote's
// step mu = tau = 1 / ||A_h|| bound; mu tau ||A_h||^2 < 1 still holds, since the
// largest eigenvalue of A_h A_h^* (the Neumann Laplacian) is below 8 / h^2.
// On grids coarser than 512^2 the schedule keeps eps_L at its 512^2 value
// instead of letting eq. stop_tol's (512 h)^2 loosen it: measured on the 128^2
// and 256^2 serving pairs, the loosened tolerance took the p = 1 error to
// 2e-4 at 128^2; the capped scales lie at or below settings measured at 5e-5
// or less.
struct CalibratedSchedule {
    double tol_scale, alpha, theta, step_ratio;
};
static constexpr CalibratedSchedule kCalibrated[2] = {{30.0, 0.5, 1.0, 1.0}, {3.0, -1.0, 1.0, 0.02}};

extern "C" w1_status w1_calibrated_schedule(int norm, double* tol_scale, double* alpha, double* theta,
                                            double* step_ratio)
{
    if (!tol_scale || !alpha || !theta || !step_ratio) return fail(W1_ERR_INVALID_ARG, "NULL output");
    if (norm == W1_NORM_L1 || norm == W1_NORM_L2) {
        const CalibratedSchedule& c = kCalibrated[norm == W1_NORM_L1 ? 0 : 1];
        *tol_scale = c.tol_scale;
        *alpha = c.alpha;
        *theta = c.theta;
        *step_ratio = c.step_ratio;
        return W1_OK;
    }
    if (norm == W1_NORM_LINF) {
        *tol_scale = 1.0;
        *alpha = -1.0;
        *theta = 0.5;
        *step_ratio = 1.0;
        return W1_OK;
    }
    return fail(W1_ERR_INVALID_ARG, "norm must be 1, 2 or 3");
}

extern "C" void w1_default_options(w1_options* o)
{
    if (!o) return;
    o->check_every = 0;
    o->max_iters = 1000000;
    o->theta = 0.5;
    o->alpha = -1.0;
    o->time_budget_s = 60.0;
    o->path = 0;
    o->rows_per_thread = 0;
    o->eager = 0;
    o->tune = 0;
    o->algorithm = 3;
    o->step_ratio = 1.0;
    o->schedule = 0;
    o->estimate = 0;
}

extern "C" const char* w1_last_error(void) { return g_err.c_str(); }

extern "C" const char* w1_status_string(w1_status s)
{
    switch (s) {
    case W1_OK: return "ok";
    case W1_ERR_INVALID_ARG: return "invalid argument";
    case W1_ERR_SHAPE: return "grid not divisible by 2^(levels-1)";
    case W1_ERR_MASS: return "mass imbalance or non-finite density";
    case W1_ERR_NOMEM: return "out of memory";
    case W1_ERR_CUDA: return "CUDA error";
    case W1_ERR_NOT_CONVERGED: return "iteration cap reached";
    case W1_ERR_TIMEOUT: return "device time budget reached";
    case W1_PENDING: return "pending";
    case W1_ERR_BUDGET: return "over the memory budget";
    case W1_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

// Carves the arena: control blocks, partials, FP64 certificate scratch, levels.
static size_t layout(w1_plan* p, char* base)
{
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        off = align_up(off, 256);
        char* r = base ? base + off : nullptr;
        off += bytes;
        return r;
    };
    const int B = p->batch;
    p->ctl = reinterpret_cast<Ctl*>(take(sizeof(Ctl) * B));
    size_t pd = final_part_doubles(B);
    if (prep_part_doubles(B) > pd) pd = prep_part_doubles(B);
    for (int l = 0; l < p->L; ++l) {
        // with tuning a level may take either streaming kernel: room for both
        if (p->lv[l].path == 2 || p->opt.tune) {
            size_t s = step_part_doubles(p->lv[l].nx, p->lv[l].ny, p->lv[l].rows, B);
            if (s > pd) pd = s;
        }
        if (p->lv[l].path == 3 || p->opt.tune) {
            size_t s = tblock_part_doubles(p->lv[l].nx, p->lv[l].ny, B);
            if (s > pd) pd = s;
        }
        if (p->lv[l].path == 4) {
            size_t s = pd_part_doubles(p->lv[l].nx, p->lv[l].ny, B);
            if (s > pd) pd = s;
        }
    }
    p->part_doubles = pd;
    p->part = reinterpret_cast<double*>(take(pd * sizeof(double)));
    const size_t n = (size_t)p->nx * p->ny;
    p->q = reinterpret_cast<double*>(take(2 * n * B * sizeof(double)));
    for (int l = 0; l < p->L; ++l) {
        LevelPlan& v = p->lv[l];
        const size_t b = (size_t)v.nx * v.ny * sizeof(float) * B;
        v.rho = reinterpret_cast<float*>(take(b));
        const int nb = ((v.path == 1 || v.path == 4) && !p->opt.tune) ? 1 : 2;
        for (int s = 0; s < 2; ++s) {
            v.m1[s] = s < nb ? reinterpret_cast<float*>(take(b)) : nullptr;
            v.m2[s] = s < nb ? reinterpret_cast<float*>(take(b)) : nullptr;
            v.phi[s] = s < nb ? reinterpret_cast<float*>(take(b)) : nullptr;
        }
        for (int k = 0; k < 6; ++k) v.pd[k] = v.path == 4 ? reinterpret_cast<float*>(take(b)) : nullptr;
        v.lam = v.path == 4 ? reinterpret_cast<float*>(take((size_t)(v.nx + v.ny) * sizeof(float))) : nullptr;
    }
    return align_up(off, 256);
}

static w1_status bind_arena(w1_plan* p, char* base, size_t bytes)
{
    if (bytes < p->ws_bytes) return fail(W1_ERR_INVALID_ARG, "workspace smaller than w1_plan_workspace_bytes");
    if (reinterpret_cast<uintptr_t>(base) % 256 != 0) return fail(W1_ERR_INVALID_ARG, "workspace not 256-byte aligned");
    layout(p, base);
    p->ws = base;
    W1_CK(cudaMemset(p->ctl, 0, sizeof(Ctl) * p->batch));
    for (int l = 0; l < p->L; ++l) {
        const LevelPlan& v = p->lv[l];
        if (v.path != 4) continue;
        std::vector<float> lam(v.nx + v.ny);
        pd_eigen(v.nx, v.h, lam.data());
        pd_eigen(v.ny, v.h, lam.data() + v.nx);
        W1_CK(cudaMemcpy(v.lam, lam.data(), lam.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
    return W1_OK;
}

// Fills every field of p that does not need device memory (levels, paths,
// tolerances, arena size).  Shared by plan creation and w1_plan_bytes.
static w1_status configure(w1_plan* p, int nx, int ny, double h, int levels, int norm, double tol, int max_batch,
                           const w1_options* opt, bool tune_now)
{
    if (nx < 1 || ny < 1) return fail(W1_ERR_INVALID_ARG, "nx and ny must be >= 1");
    if (max_batch < 1 || max_batch > 65535) return fail(W1_ERR_INVALID_ARG, "max_batch must lie in [1, 65535]");
    if (norm != W1_NORM_L1 && norm != W1_NORM_L2 && norm != W1_NORM_LINF) return fail(W1_ERR_INVALID_ARG, "norm must be 1, 2 or 3");
    w1_options o;
    w1_default_options(&o);
    if (opt) o = *opt;
    // K = 0: 32 steps between tests for Algorithm 3, 8 for Algorithm 4 (few steps
    // per level); 64 under the calibrated schedule for p = 1, 2 (a test step costs
    // several plain steps in the on-chip kernels: measured on the 512^2 reference
    // pairs, K = 64 ran 9 % faster than 32 with every error still within 2.5e-5,
    // K = 16 14 % slower)
    if (o.check_every == 0)
        o.check_every = o.algorithm == 4 ? 8 : (o.schedule == 1 && norm != W1_NORM_LINF ? 64 : 32);
    if (o.check_every < 2 || (o.check_every & 1)) return fail(W1_ERR_INVALID_ARG, "check_every must be even and >= 2");
    if (!(o.theta > 0.0) || o.theta > 1.0) return fail(W1_ERR_INVALID_ARG, "theta must lie in (0, 1]");
    if (o.max_iters < 1) return fail(W1_ERR_INVALID_ARG, "max_iters must be >= 1");
    if (o.path < 0 || o.path > 3) return fail(W1_ERR_INVALID_ARG, "path must be 0, 1, 2 or 3");
    if (o.tune < 0 || o.tune > 3) return fail(W1_ERR_INVALID_ARG, "tune must be 0, 1, 2 or 3");
    if (o.estimate < 0 || o.estimate > 1) return fail(W1_ERR_INVALID_ARG, "estimate must be 0 or 1");
    if (o.schedule < 0 || o.schedule > 1) return fail(W1_ERR_INVALID_ARG, "schedule must be 0 or 1");
    if (!(o.step_ratio > 0.0) || o.step_ratio > 1e6 || o.step_ratio < 1e-6)
        return fail(W1_ERR_INVALID_ARG, "step_ratio must lie in [1e-6, 1e6]");
    if (o.tile < 0 || o.tile > W1_TILE_VARIANTS) return fail(W1_ERR_INVALID_ARG, "tile must lie in [0, W1_TILE_VARIANTS]");
    if (o.check_every % (2 * tblock_depth(o.tile > 0 ? o.tile - 1 : 0)) != 0)
        return fail(W1_ERR_INVALID_ARG, "check_every must be a multiple of twice the temporal block depth");
    // stop tests happen every K steps, so the cap is a multiple of K
    o.max_iters = (o.max_iters + o.check_every - 1) / o.check_every * o.check_every;
    if (!(h > 0.0)) h = 1.0 / (double)(nx > ny ? nx : ny);
    if (levels <= 0) {
        // the paper's L = log2(1/h) - 3 (Sec. 5.3), kept divisible
        int L = (int)std::lround(std::log2(1.0 / h)) - 3;
        if (L < 1) L = 1;
        while (L > 1 && ((nx % (1 << (L - 1))) || (ny % (1 << (L - 1))) || (nx >> (L - 1)) < 2 ||
                         (ny >> (L - 1)) < 2))
            --L;
        levels = L;
    }
    if (levels > W1_MAX_LEVELS) return fail(W1_ERR_SHAPE, "at most 16 levels");
    const int div = 1 << (levels - 1);
    if (nx % div || ny % div) return fail(W1_ERR_SHAPE, "nx and ny must be divisible by 2^(levels-1)");
    const bool alg4 = o.algorithm == 4;
    if (o.algorithm != 0 && o.algorithm != 3 && !alg4) return fail(W1_ERR_INVALID_ARG, "algorithm must be 3 or 4");
    double tol_scale = 1.0;
    bool cap_coarse = false;  // calibrated: eps_L no looser than at h = 1/512
    if (o.schedule == 1 && !alg4 && norm != W1_NORM_LINF) {
        // calibrated schedule (w1_options.schedule): measured on the 512^2
        // ellipse-texture pairs against their converged W1 with the saddle estimate
        const CalibratedSchedule& c = kCalibrated[norm == W1_NORM_L1 ? 0 : 1];
        tol_scale = c.tol_scale;
        o.alpha = c.alpha;
        o.theta = c.theta;
        o.step_ratio = c.step_ratio;
        cap_coarse = true;
    }
    if (!(tol > 0.0)) {
        double s2 = (512.0 * h) * (512.0 * h);
        if (cap_coarse) s2 = std::min(s2, 1.0);
        tol = alg4 ? std::min(2e-4, 1e-4 / 32.0 * s2)  // eq. stop_tol, Alg. 4
                   : 1e-6 / 128.0 * s2 * tol_scale;    // eq. stop_tol, Alg. 3
    }
    int dev = 0;
    W1_CK(cudaGetDevice(&dev));
    w1_status st = prepare_device(dev);
    if (st != W1_OK) return st;
    p->device = dev;
    p->nx = nx;
    p->ny = ny;
    p->L = levels;
    p->norm = norm;
    p->batch = max_batch;
    p->h = h;
    p->tol = tol;
    p->opt = o;
    for (int l = 0; l < levels; ++l) {
        LevelPlan& v = p->lv[l];
        const int sh = levels - 1 - l;
        v.nx = nx >> sh;
        v.ny = ny >> sh;
        v.h = h * (double)(1 << sh);
        const double mu = o.theta * v.h / (2.0 * std::sqrt(2.0));  // theta / ||A_h||, ||A_h|| <= 2 sqrt(2) / h
        v.mu = (float)(mu / std::sqrt(o.step_ratio));  // mu tau = mu^2 for any ratio tau / mu
        v.tau = (float)(mu * std::sqrt(o.step_ratio));
        v.tol = tol * std::pow(v.h / h, o.alpha);  // eq. tol_formula_propose
        if (alg4) {
            // prox-PDHG: mu = tau = theta (the paper's 1/2), every level on path 4
            if (!pd_level_ok(v.nx, v.ny))
                return fail(W1_ERR_UNSUPPORTED, "Algorithm 4 needs level sides that are powers of two in [2, 1024]");
            v.mu = (float)o.theta;
            v.tau = (float)o.theta;
            v.path = 4;
            v.cluster = 0;
            v.rows = 0;
            continue;
        }
        int c = resident_cluster_for(v.nx, v.ny);
        if (c > 0 && resident_cluster_ok(norm, c, v.nx, v.ny) <= 0) c = 0;
        if (o.path == 1 && c == 0) return fail(W1_ERR_UNSUPPORTED, "level too large for the resident path");
        if (o.path == 3 && v.nx % 4 != 0) return fail(W1_ERR_UNSUPPORTED, "temporal blocking needs nx % 4 == 0");
        if (o.path == 1 || (o.path == 0 && c > 0))
            v.path = 1;
        else if (o.path == 3 || (o.path == 0 && v.nx % 4 == 0))
            v.path = 3;  // temporally blocked streaming
        else
            v.path = 2;  // one step per launch
        v.cluster = v.path == 1 ? c : 0;
        v.tile = o.tile > 0 ? o.tile - 1 : 0;
        if (o.tune && o.path == 0 && tune_now) {
            w1_level_choice ch;
            if (w1_autotune_level(v.nx, v.ny, norm, max_batch, o.tune, 128, &ch, nullptr, nullptr) == W1_OK &&
                (ch.path != 3 || o.check_every % (2 * tblock_depth(ch.tile)) == 0)) {
                v.path = ch.path;
                v.cluster = ch.path == 1 ? ch.cluster : 0;
                if (ch.path == 3 && o.tile == 0) v.tile = ch.tile;
            }
        }
        v.rows = o.rows_per_thread > 0 ? o.rows_per_thread : stream_rows_auto(v.nx, v.ny, max_batch);
    }
    p->ws_bytes = layout(p, nullptr);
    return W1_OK;
}

extern "C" size_t w1_plan_bytes(int nx, int ny, double h, int levels, int norm, double tol, int max_batch,
                                const w1_options* opt)
{
    w1_plan tmp{};
    if (configure(&tmp, nx, ny, h, levels, norm, tol, max_batch, opt, false) != W1_OK) return 0;
    return tmp.ws_bytes;
}

extern "C" w1_status w1_plan_create_batch(int nx, int ny, double h, int levels, int norm, double tol, int max_batch,
                                          const w1_options* opt, w1_plan** out)
{
    if (!out) return fail(W1_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    w1_plan* p = new (std::nothrow) w1_plan();
    if (!p) return fail(W1_ERR_NOMEM, "host allocation failed");
    w1_status st = configure(p, nx, ny, h, levels, norm, tol, max_batch, opt, true);
    if (st == W1_OK && p->lv[0].path == 4) st = pd_device_tables(p->device, &p->tw);
    if (st != W1_OK) {
        delete p;
        return st;
    }
    char* base = nullptr;
    cudaError_t e = cudaMalloc(&base, p->ws_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete p;
        return fail(W1_ERR_NOMEM, std::string("cudaMalloc workspace: ") + cudaGetErrorString(e));
    }
    st = bind_arena(p, base, p->ws_bytes);
    if (st != W1_OK) {
        cudaFree(base);
        delete p;
        return st;
    }
    p->own_ws = true;
    e = cudaMallocHost(&p->host_ctl, sizeof(Ctl) * max_batch);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->body_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cudaGetLastError();
        w1_plan_destroy(p);
        return fail(W1_ERR_CUDA, std::string("plan streams: ") + cudaGetErrorString(e));
    }
    *out = p;
    return W1_OK;
}

extern "C" w1_status w1_plan_create_ex(int nx, int ny, double h, int levels, int norm, double tol,
                                       const w1_options* opt, w1_plan** out)
{
    return w1_plan_create_batch(nx, ny, h, levels, norm, tol, 1, opt, out);
}

extern "C" w1_status w1_plan_create(int nx, int ny, double h, int levels, int norm, double tol, w1_plan** out)
{
    return w1_plan_create_batch(nx, ny, h, levels, norm, tol, 1, nullptr, out);
}

extern "C" w1_status w1_plan_destroy(w1_plan* p)
{
    if (!p) return W1_OK;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(p->device);
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    if (p->body_stream) cudaStreamDestroy(p->body_stream);
    if (p->host_ctl) cudaFreeHost(p->host_ctl);
    if (p->own_ws && p->ws) cudaFree(p->ws);
    if (p->in0) cudaFree(p->in0);
    if (p->in1) cudaFree(p->in1);
    if (p->flux_d) cudaFree(p->flux_d);
    if (p->host_done) cudaEventDestroy(p->host_done);
    cudaGetLastError();
    cudaSetDevice(cur);
    delete p;
    return W1_OK;
}

extern "C" size_t w1_plan_workspace_bytes(const w1_plan* p) { return p ? p->ws_bytes : 0; }

extern "C" int w1_plan_max_batch(const w1_plan* p) { return p ? p->batch : 0; }

extern "C" w1_status w1_plan_set_workspace(w1_plan* p, void* dev, size_t bytes)
{
    if (!p || !dev) return fail(W1_ERR_INVALID_ARG, "NULL plan or workspace");
    char* old = p->ws;
    const bool old_own = p->own_ws;
    w1_status st = bind_arena(p, static_cast<char*>(dev), bytes);
    if (st != W1_OK) {
        layout(p, old);
        p->ws = old;
        return st;
    }
    if (old_own && old) cudaFree(old);
    p->own_ws = false;
    // the graph holds the old addresses
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    p->exec = nullptr;
    p->graph = nullptr;
    p->graph_ok = false;
    return W1_OK;
}

static IterArgs iter_args(const w1_plan* p, int l)
{
    const LevelPlan& v = p->lv[l];
    IterArgs it{};
    it.nx = v.nx;
    it.ny = v.ny;
    it.mu = v.mu;
    it.tau = v.tau;
    it.ih = (float)(1.0 / v.h);
    it.h = v.h;
    it.tol = v.tol;
    it.cap = p->opt.max_iters;
    it.K = p->opt.check_every;
    it.fixed = 0;
    it.level = l;
    it.budget_ns = (unsigned long long)(p->opt.time_budget_s * 1e9);
    it.stride = (long long)v.nx * v.ny;
    it.ctl = p->ctl;
    it.fpr_out = nullptr;
    it.iters_out = nullptr;
    return it;
}

static PdArgs pd_args(const w1_plan* p, int l)
{
    const LevelPlan& v = p->lv[l];
    PdArgs a{};
    a.nx = v.nx;
    a.ny = v.ny;
    a.pairs = p->batch;
    a.mu = v.mu;
    a.tau = v.tau;
    a.ih = (float)(1.0 / v.h);
    a.h = v.h;
    a.tol = v.tol;
    a.stride = (long long)v.nx * v.ny;
    a.rho = v.rho;
    a.m1 = v.m1[0];
    a.m2 = v.m2[0];
    a.f1 = v.pd[0];
    a.f2 = v.pd[1];
    a.g1 = v.pd[2];
    a.g2 = v.pd[3];
    a.w = v.pd[4];
    a.t = v.pd[5];
    a.tw = p->tw;
    a.lamx = v.lam;
    a.lamy = v.lam + v.nx;
    a.ctl = p->ctl;
    a.part = p->part;
    a.g_out = nullptr;
    a.use_cond = 1;
    a.level = l;
    a.K = p->opt.check_every;
    a.cap = p->opt.max_iters;
    a.budget_ns = (unsigned long long)(p->opt.time_budget_s * 1e9);
    return a;
}

// Level start of a prox-PDHG level: zeros on the coarsest level, else the
// interpolation of m and of phi (both flux-like, Sec. 3.3), phibar = phi.
static cudaError_t pd_level_init(w1_plan* p, int l, cudaStream_t s)
{
    LevelPlan& v = p->lv[l];
    const int B = p->batch;
    const size_t b = (size_t)v.nx * v.ny * sizeof(float) * B;
    cudaError_t e = cudaSuccess;
    if (l == 0) {
        float* planes[6] = {v.m1[0], v.m2[0], v.pd[0], v.pd[1], v.pd[2], v.pd[3]};
        for (float* q : planes)
            if (e == cudaSuccess) e = cudaMemsetAsync(q, 0, b, s);
        return e;
    }
    const LevelPlan& c = p->lv[l - 1];
    // the third (potential) plane of the interpolation is unused here: scratch in and out
    e = launch_prolong(c.nx, c.ny, c.m1[0], c.m2[0], c.pd[4], v.m1[0], v.m2[0], v.pd[5], B, p->ctl, s);
    if (e == cudaSuccess) e = launch_prolong(c.nx, c.ny, c.pd[0], c.pd[1], c.pd[4], v.pd[0], v.pd[1], v.pd[5], B, p->ctl, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(v.pd[2], v.pd[0], b, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(v.pd[3], v.pd[1], b, cudaMemcpyDeviceToDevice, s);
    return e;
}

// Captures restriction and the level loop of Algorithm 3 into p->graph.
static w1_status build_graph(w1_plan* p)
{
    cudaStream_t s = p->cap_stream;
    const int B = p->batch;
    W1_CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
    auto abort_capture = [&](w1_status st) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(s, &g);
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return st;
    };
#define CAP_CK(call)                                                                               \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return abort_capture(fail(W1_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_))); \
    } while (0)
    for (int l = p->L - 1; l > 0; --l)
        CAP_CK(launch_restrict(p->lv[l].rho, p->lv[l].nx, p->lv[l].ny, p->lv[l - 1].rho, B, p->ctl, s));
    for (int l = 0; l < p->L; ++l) {
        LevelPlan& v = p->lv[l];
        const size_t b = (size_t)v.nx * v.ny * sizeof(float) * B;
        CAP_CK(launch_level_begin(p->ctl, l, B, s));
        if (v.path == 4) {
            CAP_CK(pd_level_init(p, l, s));
        } else if (l == 0) {
            CAP_CK(cudaMemsetAsync(v.m1[0], 0, b, s));
            CAP_CK(cudaMemsetAsync(v.m2[0], 0, b, s));
            CAP_CK(cudaMemsetAsync(v.phi[0], 0, b, s));
        } else {
            const LevelPlan& c = p->lv[l - 1];
            CAP_CK(launch_prolong(c.nx, c.ny, c.m1[0], c.m2[0], c.phi[0], v.m1[0], v.m2[0], v.phi[0], B, p->ctl, s));
        }
        if (v.path == 1) {
            ResArgs a{};
            a.drop_rank = fault_halo_rank();
            a.m1 = v.m1[0];
            a.m2 = v.m2[0];
            a.phi = v.phi[0];
            a.rho = v.rho;
            a.pairs = B;
            a.it = iter_args(p, l);
            CAP_CK(launch_resident(p->norm, v.cluster, a, s));
        } else {
            cudaStreamCaptureStatus cs;
            cudaGraph_t g = nullptr;
            const cudaGraphNode_t* deps = nullptr;
            size_t ndeps = 0;
            CAP_CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &ndeps));
            cudaGraphConditionalHandle h;
            CAP_CK(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
            alignas(cudaGraphNodeParams) unsigned char npbuf[sizeof(cudaGraphNodeParams)];
            std::memset(npbuf, 0, sizeof(npbuf));
            cudaGraphNodeParams& np = *reinterpret_cast<cudaGraphNodeParams*>(npbuf);
            np.type = cudaGraphNodeTypeConditional;
            np.conditional.handle = h;
            np.conditional.type = cudaGraphCondTypeWhile;
            np.conditional.size = 1;
            cudaGraphNode_t node;
            CAP_CK(cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &np));
            cudaGraph_t body = np.conditional.phGraph_out[0];
            CAP_CK(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
            CAP_CK(cudaStreamBeginCaptureToGraph(p->body_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
            const int K = p->opt.check_every;
            const int per = v.path == 3 ? tblock_depth(v.tile) : 1;  // steps per launch
            const int nl = K / per;                             // launches per body (even: K and per are)
            cudaError_t e = cudaSuccess;
            if (v.path == 4) {
                const PdArgs pa = pd_args(p, l);
                for (int k = 0; k < K && e == cudaSuccess; ++k) e = launch_pd_step(p->norm, k == K - 1, pa, p->body_stream);
            }
            for (int k = 0; k < nl && e == cudaSuccess && v.path != 4; ++k) {
                StepArgs a{};
                const int src = k & 1, dst = src ^ 1;
                a.m1 = v.m1[src];
                a.m2 = v.m2[src];
                a.phi = v.phi[src];
                a.rho = v.rho;
                a.m1o = v.m1[dst];
                a.m2o = v.m2[dst];
                a.phio = v.phi[dst];
                a.rows = v.rows;
                a.pairs = B;
                a.it = iter_args(p, l);
                a.part = p->part;
                a.use_cond = 1;
                a.tile = v.tile;
                e = v.path == 3 ? launch_tblock(p->norm, k == nl - 1, a, p->body_stream)
                                : launch_step(p->norm, k == nl - 1, a, p->body_stream);
            }
            if (e == cudaSuccess) e = launch_decide(p->ctl, B, h, p->body_stream);
            if (e != cudaSuccess) {
                cudaGraph_t bg;
                cudaStreamEndCapture(p->body_stream, &bg);
                return abort_capture(fail(W1_ERR_CUDA, std::string("capture step: ") + cudaGetErrorString(e)));
            }
            cudaGraph_t bg = nullptr;
            CAP_CK(cudaStreamEndCapture(p->body_stream, &bg));
        }
    }
    if (p->lv[p->L - 1].path == 4)  // the Kantorovich potential from phi (Appendix B)
        CAP_CK(launch_pd_potential(pd_args(p, p->L - 1), p->lv[p->L - 1].phi[0], s));
#undef CAP_CK
    cudaGraph_t g = nullptr;
    W1_CK(cudaStreamEndCapture(s, &g));
    p->graph = g;
    W1_CK(cudaGraphInstantiate(&p->exec, g, 0));
    p->graph_ok = true;
    return W1_OK;
}

static w1_status pair_status(const w1_plan* p, const Ctl* c)
{
    if (c->error == 1) return W1_ERR_MASS;
    if (c->timeout) return W1_ERR_TIMEOUT;
    for (int l = 0; l < p->L; ++l)
        if (!c->conv[l]) return W1_ERR_NOT_CONVERGED;
    return W1_OK;
}

static void fill_stats(const w1_plan* p, const Ctl* c, w1_stats* st)
{
    std::memset(st, 0, sizeof(*st));
    st->levels = p->L;
    int conv = 1;
    for (int l = 0; l < p->L; ++l) {
        st->nx[l] = p->lv[l].nx;
        st->ny[l] = p->lv[l].ny;
        st->iters[l] = c->iters[l];
        st->fpr[l] = c->fpr[l];
        st->tol[l] = p->lv[l].tol;
        st->path[l] = p->lv[l].path;
        st->cluster[l] = p->lv[l].path == 3 ? p->lv[l].tile + 1 : p->lv[l].cluster;
        conv &= c->conv[l] ? 1 : 0;
    }
    st->w1 = p->opt.estimate == 1 ? c->f : c->saddle;
    st->primal = c->f;
    st->saddle = c->saddle;
    st->dual = c->dual;
    st->lb = c->lb;
    st->ub = c->ub;
    st->route = c->route;
    st->res_l1 = c->res_l1;
    st->rho_l1 = c->rho_l1;
    st->gmax = c->gmax;
    st->mass0 = c->mass0;
    st->mass1 = c->mass1;
    st->mass_shift = c->mean;
    st->converged = conv && !c->error && !c->timeout;
}

// The level sequence of build_graph, launched directly on s.  Streaming levels
// test convergence on the host after every K steps (one small copy and a
// stream synchronisation per test), so this mode is for profiling only.
static w1_status run_eager(w1_plan* p, cudaStream_t s)
{
    const int B = p->batch;
    for (int l = p->L - 1; l > 0; --l)
        W1_CK(launch_restrict(p->lv[l].rho, p->lv[l].nx, p->lv[l].ny, p->lv[l - 1].rho, B, p->ctl, s));
    std::vector<Ctl> host(B);
    for (int l = 0; l < p->L; ++l) {
        LevelPlan& v = p->lv[l];
        NvtxRange range("w1 level %d %dx%d path %d", l, v.nx, v.ny, v.path);
        const size_t b = (size_t)v.nx * v.ny * sizeof(float) * B;
        W1_CK(launch_level_begin(p->ctl, l, B, s));
        if (v.path == 4) {
            W1_CK(pd_level_init(p, l, s));
        } else if (l == 0) {
            W1_CK(cudaMemsetAsync(v.m1[0], 0, b, s));
            W1_CK(cudaMemsetAsync(v.m2[0], 0, b, s));
            W1_CK(cudaMemsetAsync(v.phi[0], 0, b, s));
        } else {
            const LevelPlan& c = p->lv[l - 1];
            W1_CK(launch_prolong(c.nx, c.ny, c.m1[0], c.m2[0], c.phi[0], v.m1[0], v.m2[0], v.phi[0], B, p->ctl, s));
        }
        if (v.path == 1) {
            ResArgs a{};
            a.drop_rank = fault_halo_rank();
            a.m1 = v.m1[0];
            a.m2 = v.m2[0];
            a.phi = v.phi[0];
            a.rho = v.rho;
            a.pairs = B;
            a.it = iter_args(p, l);
            W1_CK(launch_resident(p->norm, v.cluster, a, s));
            continue;
        }
        const int K = p->opt.check_every;
        const int per = v.path == 3 ? tblock_depth(v.tile) : 1;
        const int nl = K / per;
        for (;;) {
            if (v.path == 4) {
                const PdArgs pa = pd_args(p, l);
                for (int k = 0; k < K; ++k) W1_CK(launch_pd_step(p->norm, k == K - 1, pa, s));
            }
            for (int k = 0; k < nl && v.path != 4; ++k) {
                StepArgs a{};
                const int src = k & 1, dst = src ^ 1;
                a.m1 = v.m1[src];
                a.m2 = v.m2[src];
                a.phi = v.phi[src];
                a.rho = v.rho;
                a.m1o = v.m1[dst];
                a.m2o = v.m2[dst];
                a.phio = v.phi[dst];
                a.rows = v.rows;
                a.pairs = B;
                a.it = iter_args(p, l);
                a.part = p->part;
                a.use_cond = 1;
                a.tile = v.tile;
                W1_CK(v.path == 3 ? launch_tblock(p->norm, k == nl - 1, a, s) : launch_step(p->norm, k == nl - 1, a, s));
            }
            W1_CK(cudaMemcpyAsync(host.data(), p->ctl, sizeof(Ctl) * B, cudaMemcpyDeviceToHost, s));
            W1_CK(cudaStreamSynchronize(s));
            bool any = false;
            for (int q = 0; q < B; ++q) any |= host[q].active != 0;
            if (!any) break;
        }
    }
    if (p->lv[p->L - 1].path == 4) W1_CK(launch_pd_potential(pd_args(p, p->L - 1), p->lv[p->L - 1].phi[0], s));
    return W1_OK;
}

// Enqueues one batched solve on s: prep -> graph -> final statistics -> flux
// copy -> device-to-host copy of the control blocks into the plan's pinned
// result block.  Nothing waits.
static w1_status enqueue(w1_plan* p, int nbatch, const float* rho0, const float* rho1, cudaStream_t s, float* flux)
{
    NvtxRange range("w1 solve %dx%d p%d x%d", p->nx, p->ny, p->norm, nbatch);
    if (!p->opt.eager && !p->graph_ok) {
        w1_status st = build_graph(p);
        if (st != W1_OK) return st;
    }
    const long long n = (long long)p->nx * p->ny;
    const int B = p->batch;
    const LevelPlan& f = p->lv[p->L - 1];
    W1_CK(launch_prep(rho0, rho1, n, nbatch, B, p->h, p->ctl, p->part, f.rho, s));
    if (p->opt.eager) {
        w1_status st = run_eager(p, s);
        if (st != W1_OK) return st;
    } else {
        W1_CK(cudaGraphLaunch(p->exec, s));
    }
    W1_CK(launch_final(p->norm, f.m1[0], f.m2[0], f.phi[0], f.rho, f.nx, f.ny, f.h, p->q, p->part, p->ctl, B, s));
    if (flux) {
        // flux[b] = (m1 of pair b, m2 of pair b)
        W1_CK(cudaMemcpy2DAsync(flux, 2 * n * sizeof(float), f.m1[0], n * sizeof(float), n * sizeof(float), nbatch,
                                cudaMemcpyDeviceToDevice, s));
        W1_CK(cudaMemcpy2DAsync(flux + n, 2 * n * sizeof(float), f.m2[0], n * sizeof(float), n * sizeof(float),
                                nbatch, cudaMemcpyDeviceToDevice, s));
    }
    W1_CK(cudaMemcpyAsync(p->host_ctl, p->ctl, sizeof(Ctl) * nbatch, cudaMemcpyDeviceToHost, s));
    p->last_batch = nbatch;
    return W1_OK;
}

// Reads the pinned result block of the last enqueued solve (the stream must
// have passed its end).
static w1_status results(w1_plan* p, double* dist, w1_stats* stats, int* status)
{
    const int nbatch = p->last_batch;
    w1_status worst = W1_OK;
    for (int b = 0; b < nbatch; ++b) {
        const Ctl* c = p->host_ctl + b;
        if (stats) fill_stats(p, c, &stats[b]);
        const w1_status sb = pair_status(p, c);
        if (dist) dist[b] = sb == W1_ERR_MASS ? NAN : (p->opt.estimate == 1 ? c->f : c->saddle);
        if (status) status[b] = sb;
        if (worst == W1_OK && sb != W1_OK) worst = sb;
    }
    if (worst == W1_ERR_MASS) return fail(worst, "densities have different mass or a non-finite value");
    if (worst == W1_ERR_TIMEOUT) return fail(worst, "a level hit the device time budget");
    if (worst == W1_ERR_NOT_CONVERGED) return fail(worst, "a level hit max_iters");
    return W1_OK;
}

static w1_status solve_device(w1_plan* p, int nbatch, const float* rho0, const float* rho1, cudaStream_t s,
                              double* dist, float* flux, w1_stats* stats, int* status)
{
    w1_status st = enqueue(p, nbatch, rho0, rho1, s, flux);
    if (st != W1_OK) return st;
    W1_CK(cudaStreamSynchronize(s));
    return results(p, dist, stats, status);
}

extern "C" w1_status w1_solve_async(w1_plan* p, int nbatch, const float* rho0, const float* rho1, void* stream,
                                    float* flux)
{
    if (!p || !rho0 || !rho1) return fail(W1_ERR_INVALID_ARG, "NULL plan or density");
    if (nbatch < 1 || nbatch > p->batch) return fail(W1_ERR_INVALID_ARG, "batch must lie in [1, max_batch]");
    W1_CK(cudaSetDevice(p->device));
    return enqueue(p, nbatch, rho0, rho1, static_cast<cudaStream_t>(stream), flux);
}

extern "C" w1_status w1_plan_results(w1_plan* p, double* dist, w1_stats* stats, int* status)
{
    if (!p) return fail(W1_ERR_INVALID_ARG, "NULL plan");
    if (p->last_batch < 1) return fail(W1_ERR_INVALID_ARG, "no solve was enqueued on this plan");
    return results(p, dist, stats, status);
}

extern "C" w1_status w1_solve_batch(w1_plan* p, int nbatch, const float* rho0, const float* rho1, void* stream,
                                    double* dist, float* flux, w1_stats* stats, int* status)
{
    if (!p || !rho0 || !rho1 || !dist) return fail(W1_ERR_INVALID_ARG, "NULL plan, density or dist");
    if (nbatch < 1 || nbatch > p->batch) return fail(W1_ERR_INVALID_ARG, "batch must lie in [1, max_batch]");
    W1_CK(cudaSetDevice(p->device));
    return solve_device(p, nbatch, rho0, rho1, static_cast<cudaStream_t>(stream), dist, flux, stats, status);
}

extern "C" w1_status w1_solve(w1_plan* p, const float* rho0, const float* rho1, void* stream, double* dist,
                              float* flux, w1_stats* stats)
{
    return w1_solve_batch(p, 1, rho0, rho1, stream, dist, flux, stats, nullptr);
}

extern "C" w1_status w1_solve_batch_host(w1_plan* p, int nbatch, const float* rho0, const float* rho1, void* stream,
                                         double* dist, float* flux, w1_stats* stats, int* status)
{
    if (!p || !rho0 || !rho1 || !dist) return fail(W1_ERR_INVALID_ARG, "NULL plan, density or dist");
    if (nbatch < 1 || nbatch > p->batch) return fail(W1_ERR_INVALID_ARG, "batch must lie in [1, max_batch]");
    W1_CK(cudaSetDevice(p->device));
    const size_t n = (size_t)p->nx * p->ny;
    const size_t bytes = n * sizeof(float) * p->batch;
    if (!p->in0) W1_CK(cudaMalloc(&p->in0, bytes));
    if (!p->in1) W1_CK(cudaMalloc(&p->in1, bytes));
    if (flux && !p->flux_d) W1_CK(cudaMalloc(&p->flux_d, 2 * bytes));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // Host-buffer calls are the ones a service issues from many host threads at
    // once; a thread that spins in the driver until its solve ends takes a core
    // from the threads that still submit work, so this call waits asleep.
    if (!p->host_done) W1_CK(cudaEventCreateWithFlags(&p->host_done, cudaEventBlockingSync | cudaEventDisableTiming));
    W1_CK(cudaMemcpyAsync(p->in0, rho0, n * sizeof(float) * nbatch, cudaMemcpyHostToDevice, s));
    W1_CK(cudaMemcpyAsync(p->in1, rho1, n * sizeof(float) * nbatch, cudaMemcpyHostToDevice, s));
    w1_status st = enqueue(p, nbatch, p->in0, p->in1, s, flux ? p->flux_d : nullptr);
    if (st == W1_OK) {
        W1_CK(cudaEventRecord(p->host_done, s));
        W1_CK(cudaEventSynchronize(p->host_done));
        st = results(p, dist, stats, status);
    }
    if (flux && st != W1_ERR_CUDA && st != W1_ERR_NOMEM && st != W1_ERR_INVALID_ARG) {
        W1_CK(cudaMemcpyAsync(flux, p->flux_d, 2 * n * sizeof(float) * nbatch, cudaMemcpyDeviceToHost, s));
        W1_CK(cudaStreamSynchronize(s));
    }
    return st;
}

extern "C" w1_status w1_solve_host(w1_plan* p, const float* rho0, const float* rho1, void* stream, double* dist,
                                   float* flux, w1_stats* stats)
{
    return w1_solve_batch_host(p, 1, rho0, rho1, stream, dist, flux, stats, nullptr);
}

extern "C" w1_status w1_plan_potential(w1_plan* p, float* phi, void* stream)
{
    if (!p || !phi) return fail(W1_ERR_INVALID_ARG, "NULL plan or phi");
    W1_CK(cudaSetDevice(p->device));
    const LevelPlan& f = p->lv[p->L - 1];
    const int nb = p->last_batch > 0 ? p->last_batch : 1;
    W1_CK(cudaMemcpyAsync(phi, f.phi[0], (size_t)f.nx * f.ny * sizeof(float) * nb, cudaMemcpyDeviceToDevice,
                          static_cast<cudaStream_t>(stream)));
    return W1_OK;
}

// ---------------------------------------------------------------------------
// Mixed-size batches
// ---------------------------------------------------------------------------
//
// One batched plan per size class holds that class's arena (levels, control
// blocks, partials).  Classes whose every level fits one CTA run together in one
// persistent launch (k_cascade: a CTA takes a pair, runs all its levels, takes
// the next; pairs of the largest grids first).  When some class has a level
// that needs a cluster of CASCADE_CLUSTER CTAs (and fits one), the persistent
// launch runs in clusters instead (k_cascade_cl): clusters take those pairs
// first, then each CTA takes single-CTA pairs alone.  Classes that fit neither
// run their own plan's graph on a stream of their own.  A solve is: record -> [other classes on
// their streams] and [prep per class -> graph: restriction per class -> the
// persistent launch -> final statistics and the read-back per class] -> join.

struct w1_mixed {
    int device, n, norm;
    std::vector<w1_plan*> plans;
    std::vector<int> count;
    std::vector<int> persistent;   // 1: the class runs in the persistent launch
    std::vector<int> order;        // persistent single-CTA classes, largest grid first
    std::vector<int> order_big;    // persistent cluster classes, largest grid first
    CascadeClass* d_cls;
    CascadeClass* d_big;
    CascadeClass* d_all;           // every persistent class, for the coarse launch
    unsigned int* d_next;          // work counters: single-CTA pairs, cluster pairs, coarse launch
    int ctas, total, total_big;
    int coarse_ctas;               // > 0: the coarse launch runs first
    int side_ctas;                 // > 0: single-CTA persistent CTAs beside the cluster launch
    bool fine_work;                // some class has a level beyond the coarse launch
    cudaStream_t side;             // their stream (forked from the solve's stream and joined back)
    cudaEvent_t fork, join;
    int clusters;                  // > 0: the persistent launch runs in clusters (some class needs one)
    bool wide;                     // the persistent launch's level layout
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> done;
    cudaEvent_t start;
    cudaStream_t cap_stream;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    bool eager;
};

// restriction of every persistent class -> the persistent launch -> final
// statistics and read-back of every persistent class, enqueued on s
static w1_status mixed_sequence(w1_mixed* m, cudaStream_t s)
{
    if (m->total + m->total_big == 0) return W1_OK;
    W1_CK(cudaMemsetAsync(m->d_next, 0, 3 * sizeof(unsigned int), s));
    std::vector<int> all(m->order_big);
    all.insert(all.end(), m->order.begin(), m->order.end());
    for (int c : all) {
        w1_plan* p = m->plans[c];
        for (int l = p->L - 1; l > 0; --l)
            W1_CK(launch_restrict(p->lv[l].rho, p->lv[l].nx, p->lv[l].ny, p->lv[l - 1].rho, p->batch, p->ctl, s));
    }
    CascadeArgs a{};
    a.cls = m->d_cls;
    a.n_classes = (int)m->order.size();
    a.total = m->total;
    a.next = m->d_next;
    a.big = m->d_big;
    a.n_big = (int)m->order_big.size();
    a.total_big = m->total_big;
    a.next_big = m->d_next + 1;
    const w1_options& o = m->plans[all[0]]->opt;
    a.cap = o.max_iters;
    a.K = o.check_every;
    a.budget_ns = (unsigned long long)(o.time_budget_s * 1e9);
    if (m->coarse_ctas > 0) {
        CascadeArgs c = a;
        c.cls = m->d_all;
        c.n_classes = (int)all.size();
        c.total = m->total + m->total_big;
        c.next = m->d_next + 2;
        c.big = nullptr;
        c.n_big = 0;
        c.total_big = 0;
        c.next_big = nullptr;
        W1_CK(launch_cascade_coarse(m->norm, c, m->coarse_ctas, s));
    }
    if (m->fine_work) {
        if (m->clusters > 0) {
            // SMs that no whole cluster can use run single-CTA persistent CTAs,
            // which draw single-CTA pairs from the same counter as the clusters'
            // second phase
            const bool side = m->side_ctas > 0 && a.total > 0;
            if (side) {
                W1_CK(cudaEventRecord(m->fork, s));
                W1_CK(cudaStreamWaitEvent(m->side, m->fork, 0));
            }
            W1_CK(launch_cascade_cluster(m->norm, a, m->clusters, s));
            if (side) {
                W1_CK(launch_cascade(m->norm, m->wide, a, m->side_ctas, m->side));
                W1_CK(cudaEventRecord(m->join, m->side));
                W1_CK(cudaStreamWaitEvent(s, m->join, 0));
            }
        } else {
            W1_CK(launch_cascade(m->norm, m->wide, a, m->ctas, s));
        }
    }
    for (int c : all) {
        w1_plan* p = m->plans[c];
        const LevelPlan& f = p->lv[p->L - 1];
        W1_CK(launch_final(p->norm, f.m1[0], f.m2[0], f.phi[0], f.rho, f.nx, f.ny, f.h, p->q, p->part, p->ctl,
                           p->batch, s));
        W1_CK(cudaMemcpyAsync(p->host_ctl, p->ctl, sizeof(Ctl) * p->batch, cudaMemcpyDeviceToHost, s));
    }
    return W1_OK;
}

extern "C" w1_status w1_mixed_destroy(w1_mixed* m)
{
    if (!m) return W1_OK;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(m->device);
    for (w1_plan* p : m->plans) w1_plan_destroy(p);
    for (cudaStream_t s : m->streams)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : m->done)
        if (e) cudaEventDestroy(e);
    if (m->start) cudaEventDestroy(m->start);
    if (m->exec) cudaGraphExecDestroy(m->exec);
    if (m->graph) cudaGraphDestroy(m->graph);
    if (m->cap_stream) cudaStreamDestroy(m->cap_stream);
    if (m->side) cudaStreamDestroy(m->side);
    if (m->fork) cudaEventDestroy(m->fork);
    if (m->join) cudaEventDestroy(m->join);
    if (m->d_cls) cudaFree(m->d_cls);
    if (m->d_big) cudaFree(m->d_big);
    if (m->d_all) cudaFree(m->d_all);
    if (m->d_next) cudaFree(m->d_next);
    cudaGetLastError();
    cudaSetDevice(cur);
    delete m;
    return W1_OK;
}

extern "C" w1_status w1_mixed_create(int n_classes, const int* nx, const int* ny, const int* count, int norm,
                                     double tol, const w1_options* opt, w1_mixed** out)
{
    if (!out) return fail(W1_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_classes < 1 || n_classes > 64 || !nx || !ny || !count)
        return fail(W1_ERR_INVALID_ARG, "need 1..64 size classes with nx, ny and count");
    for (int c = 0; c < n_classes; ++c)
        if (count[c] < 1) return fail(W1_ERR_INVALID_ARG, "every class needs at least one pair");
    w1_mixed* m = new (std::nothrow) w1_mixed();
    if (!m) return fail(W1_ERR_NOMEM, "host allocation failed");
    m->n = n_classes;
    m->norm = norm;
    m->eager = opt && opt->eager;
    cudaGetDevice(&m->device);
    for (int c = 0; c < n_classes; ++c) {
        w1_plan* p = nullptr;
        w1_status st = w1_plan_create_batch(nx[c], ny[c], 0.0, 0, norm, tol, count[c], opt, &p);
        if (st != W1_OK) {
            const std::string msg = g_err;
            w1_mixed_destroy(m);
            return fail(st, "class " + std::to_string(c) + ": " + msg);
        }
        m->plans.push_back(p);
        m->count.push_back(count[c]);
        // 1: every level fits the four-nodes-per-thread layout; 2: some level needs
        // the wide one; 3: some level needs a cluster of CASCADE_CLUSTER CTAs and
        // every level fits one; 0: some level fits none of these (or a path is forced)
        int kind = (opt && (opt->path != 0 || opt->algorithm == 4)) ? 0 : 1;
        for (int l = 0; l < p->L && kind; ++l) {
            const int f = cascade_level_fits(p->lv[l].nx, p->lv[l].ny);
            if (f == 0) kind = cascade_level_mode_cluster(p->lv[l].nx, p->lv[l].ny) ? 3 : 0;
            else if (!(f & 1) && kind == 1) kind = 2;
        }
        if (kind == 3)  // every level of a cluster class must have a cluster mode
            for (int l = 0; l < p->L; ++l)
                if (!cascade_level_mode_cluster(p->lv[l].nx, p->lv[l].ny)) kind = 0;
        m->persistent.push_back(kind);
    }
    m->wide = false;
    bool any_big = false;
    for (int c = 0; c < n_classes; ++c) {
        if (m->persistent[c] == 2) m->wide = true;
        if (m->persistent[c] == 3) any_big = true;
    }
    // persistent classes, largest grid first
    auto by_size = [&](std::vector<int>& ord) {
        for (size_t a = 0; a < ord.size(); ++a)
            for (size_t b = a + 1; b < ord.size(); ++b) {
                const w1_plan* pa = m->plans[ord[a]];
                const w1_plan* pb = m->plans[ord[b]];
                if ((long long)pb->nx * pb->ny > (long long)pa->nx * pa->ny) std::swap(ord[a], ord[b]);
            }
    };
    for (int c = 0; c < n_classes; ++c) {
        if (m->persistent[c] == 3) m->order_big.push_back(c);
        else if (m->persistent[c]) m->order.push_back(c);
        m->persistent[c] = m->persistent[c] ? 1 : 0;
    }
    by_size(m->order);
    by_size(m->order_big);
    auto classes_of = [&](const std::vector<int>& ord, bool big, int& total) {
        std::vector<CascadeClass> out;
        for (int c : ord) {
            const w1_plan* p = m->plans[c];
            CascadeClass k{};
            k.levels = p->L;
            k.count = p->batch;
            k.ctl = p->ctl;
            k.split = 0;
            while (k.split < p->L && (long long)p->lv[k.split].nx * p->lv[k.split].ny <= CASCADE_COARSE_NODES &&
                   p->lv[k.split].nx % 4 == 0)
                ++k.split;
            for (int l = 0; l < p->L; ++l) {
                const LevelPlan& v = p->lv[l];
                CascadeLevel& d = k.lv[l];
                d.nx = v.nx;
                d.ny = v.ny;
                d.mode = big ? cascade_level_mode_cluster(v.nx, v.ny) : 0;
                d.mu = v.mu;
                d.tau = v.tau;
                d.ih = (float)(1.0 / v.h);
                d.h = v.h;
                d.tol = v.tol;
                d.rho = v.rho;
                d.m1 = v.m1[0];
                d.m2 = v.m2[0];
                d.phi = v.phi[0];
            }
            out.push_back(k);
            total += p->batch;
        }
        return out;
    };
    std::vector<CascadeClass> cls = classes_of(m->order, false, m->total);
    std::vector<CascadeClass> big = classes_of(m->order_big, true, m->total_big);
    std::vector<CascadeClass> allc(big);
    allc.insert(allc.end(), cls.begin(), cls.end());
    bool any_coarse = false;
    for (const CascadeClass& k : allc) {
        if (k.split > 0) any_coarse = true;
        if (k.split < k.levels) m->fine_work = true;
    }
    cudaError_t e = cudaSuccess;
    if (!cls.empty() || !big.empty()) {
        if (any_big) {
            m->clusters = cascade_clusters(norm);
            if (m->clusters < 1) {
                w1_mixed_destroy(m);
                return fail(W1_ERR_CUDA, "the cluster persistent launch cannot be resident");
            }
            int dev = 0, sms = 0;
            if (!cls.empty() && cudaGetDevice(&dev) == cudaSuccess &&
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess) {
                const int left = sms - CASCADE_CLUSTER * m->clusters;
                const int fit = cascade_ctas(norm, m->wide);
                m->side_ctas = left > 0 ? std::min(left, fit) : 0;
            }
            cudaGetLastError();
            if (m->side_ctas > 0) {
                e = cudaStreamCreateWithFlags(&m->side, cudaStreamNonBlocking);
                if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m->fork, cudaEventDisableTiming);
                if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m->join, cudaEventDisableTiming);
                if (e != cudaSuccess) {
                    cudaGetLastError();
                    w1_mixed_destroy(m);
                    return fail(W1_ERR_CUDA, std::string("side stream: ") + cudaGetErrorString(e));
                }
            }
        } else {
            m->ctas = cascade_ctas(norm, m->wide);
            if (m->ctas < 1) {
                w1_mixed_destroy(m);
                return fail(W1_ERR_CUDA, "the persistent launch cannot be resident");
            }
        }
        if (!cls.empty()) {
            e = cudaMalloc(&m->d_cls, sizeof(CascadeClass) * cls.size());
            if (e == cudaSuccess)
                e = cudaMemcpy(m->d_cls, cls.data(), sizeof(CascadeClass) * cls.size(), cudaMemcpyHostToDevice);
        }
        if (e == cudaSuccess && !big.empty()) {
            e = cudaMalloc(&m->d_big, sizeof(CascadeClass) * big.size());
            if (e == cudaSuccess)
                e = cudaMemcpy(m->d_big, big.data(), sizeof(CascadeClass) * big.size(), cudaMemcpyHostToDevice);
        }
        if (e == cudaSuccess && any_coarse) {
            m->coarse_ctas = cascade_coarse_ctas(norm);
            if (m->coarse_ctas < 1) {
                w1_mixed_destroy(m);
                return fail(W1_ERR_CUDA, "the coarse launch cannot be resident");
            }
            e = cudaMalloc(&m->d_all, sizeof(CascadeClass) * allc.size());
            if (e == cudaSuccess)
                e = cudaMemcpy(m->d_all, allc.data(), sizeof(CascadeClass) * allc.size(), cudaMemcpyHostToDevice);
        }
        if (e == cudaSuccess) e = cudaMalloc(&m->d_next, 3 * sizeof(unsigned int));
    }
    m->streams.assign(n_classes, nullptr);
    m->done.assign(n_classes, nullptr);
    for (int c = 0; c < n_classes && e == cudaSuccess; ++c) {
        if (m->persistent[c]) continue;
        e = cudaStreamCreateWithFlags(&m->streams[c], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m->done[c], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m->start, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&m->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cudaGetLastError();
        w1_mixed_destroy(m);
        return fail(W1_ERR_CUDA, std::string("mixed batch set-up: ") + cudaGetErrorString(e));
    }
    if ((!cls.empty() || !big.empty()) && !m->eager) {
        // the persistent part as one CUDA graph
        W1_CK(cudaStreamBeginCapture(m->cap_stream, cudaStreamCaptureModeRelaxed));
        w1_status st = mixed_sequence(m, m->cap_stream);
        cudaGraph_t g = nullptr;
        cudaError_t ce = cudaStreamEndCapture(m->cap_stream, &g);
        if (st != W1_OK || ce != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            w1_mixed_destroy(m);
            return st != W1_OK ? st : fail(W1_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(ce));
        }
        m->graph = g;
        e = cudaGraphInstantiate(&m->exec, g, 0);
        if (e != cudaSuccess) {
            cudaGetLastError();
            w1_mixed_destroy(m);
            return fail(W1_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e));
        }
    }
    *out = m;
    return W1_OK;
}

extern "C" w1_status w1_mixed_launch_info(const w1_mixed* m, int* ctas, int* clusters, int* coarse_ctas)
{
    if (!m) return fail(W1_ERR_INVALID_ARG, "NULL batch");
    if (ctas) *ctas = m->clusters > 0 ? m->side_ctas : m->ctas;
    if (clusters) *clusters = m->clusters;
    if (coarse_ctas) *coarse_ctas = m->coarse_ctas;
    return W1_OK;
}

extern "C" int w1_mixed_persistent(const w1_mixed* m, int cls)
{
    if (!m || cls < 0 || cls >= m->n) return -1;
    return m->persistent[cls];
}

extern "C" w1_status w1_mixed_solve_async(w1_mixed* m, const float* const* rho0, const float* const* rho1,
                                          void* stream)
{
    if (!m || !rho0 || !rho1) return fail(W1_ERR_INVALID_ARG, "NULL batch or densities");
    for (int c = 0; c < m->n; ++c)
        if (!rho0[c] || !rho1[c]) return fail(W1_ERR_INVALID_ARG, "NULL density of class " + std::to_string(c));
    W1_CK(cudaSetDevice(m->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    W1_CK(cudaEventRecord(m->start, s));
    for (int c = 0; c < m->n; ++c) {
        if (m->persistent[c]) continue;
        W1_CK(cudaStreamWaitEvent(m->streams[c], m->start, 0));
        w1_status st = enqueue(m->plans[c], m->count[c], rho0[c], rho1[c], m->streams[c], nullptr);
        if (st != W1_OK) return st;
        W1_CK(cudaEventRecord(m->done[c], m->streams[c]));
    }
    std::vector<int> all(m->order_big);
    all.insert(all.end(), m->order.begin(), m->order.end());
    for (int c : all) {
        w1_plan* p = m->plans[c];
        W1_CK(launch_prep(rho0[c], rho1[c], (long long)p->nx * p->ny, p->batch, p->batch, p->h, p->ctl, p->part,
                          p->lv[p->L - 1].rho, s));
        p->last_batch = p->batch;
    }
    if (!all.empty()) {
        if (m->eager) {
            w1_status st = mixed_sequence(m, s);
            if (st != W1_OK) return st;
        } else {
            W1_CK(cudaGraphLaunch(m->exec, s));
        }
    }
    for (int c = 0; c < m->n; ++c)
        if (!m->persistent[c]) W1_CK(cudaStreamWaitEvent(s, m->done[c], 0));
    return W1_OK;
}

extern "C" w1_status w1_mixed_results(w1_mixed* m, int cls, double* dist, w1_stats* stats, int* status)
{
    if (!m || cls < 0 || cls >= m->n) return fail(W1_ERR_INVALID_ARG, "NULL batch or class out of range");
    if (m->plans[cls]->last_batch < 1) return fail(W1_ERR_INVALID_ARG, "no solve was enqueued on this batch");
    return results(m->plans[cls], dist, stats, status);
}

// ---------------------------------------------------------------------------
// Building blocks
// ---------------------------------------------------------------------------

namespace {

// Scratch of a building-block prox-PDHG call: residual, transpose, eigenvalues,
// partials, result.
struct PdScratch {
    float* w = nullptr;
    float* t = nullptr;
    float* lam = nullptr;
    double* part = nullptr;
    double* g = nullptr;
    Ctl* ctl = nullptr;
    ~PdScratch()
    {
        cudaFree(w);
        cudaFree(t);
        cudaFree(lam);
        cudaFree(part);
        cudaFree(g);
        cudaFree(ctl);
    }
};

w1_status pd_scratch(PdScratch& sc, PdArgs& a, int nx, int ny, double h)
{
    const size_t n = (size_t)nx * ny;
    W1_CK(cudaMalloc(&sc.w, n * sizeof(float)));
    W1_CK(cudaMalloc(&sc.t, n * sizeof(float)));
    W1_CK(cudaMalloc(&sc.lam, (size_t)(nx + ny) * sizeof(float)));
    W1_CK(cudaMalloc(&sc.part, pd_part_doubles(nx, ny, 1) * sizeof(double)));
    W1_CK(cudaMalloc(&sc.g, sizeof(double)));
    W1_CK(cudaMalloc(&sc.ctl, sizeof(Ctl)));
    W1_CK(cudaMemset(sc.ctl, 0, sizeof(Ctl)));
    std::vector<float> lam(nx + ny);
    pd_eigen(nx, h, lam.data());
    pd_eigen(ny, h, lam.data() + nx);
    W1_CK(cudaMemcpy(sc.lam, lam.data(), lam.size() * sizeof(float), cudaMemcpyHostToDevice));
    a.nx = nx;
    a.ny = ny;
    a.pairs = 1;
    a.h = h;
    a.ih = (float)(1.0 / h);
    a.stride = (long long)n;
    a.w = sc.w;
    a.t = sc.t;
    a.lamx = sc.lam;
    a.lamy = sc.lam + nx;
    a.part = sc.part;
    a.g_out = sc.g;
    a.ctl = sc.ctl;  // the test step's reduction counter
    a.use_cond = 0;
    return W1_OK;
}

}  // namespace

extern "C" w1_status w1_poisson(int nx, int ny, double h, const float* r, float* psi, void* stream)
{
    if (!r || !psi || !(h > 0.0)) return fail(W1_ERR_INVALID_ARG, "bad arguments to w1_poisson");
    if (!pd_level_ok(nx, ny)) return fail(W1_ERR_UNSUPPORTED, "nx and ny must be powers of two in [2, 1024]");
    int dev = 0;
    W1_CK(cudaGetDevice(&dev));
    w1_status st = prepare_device(dev);
    if (st != W1_OK) return st;
    PdArgs a{};
    st = pd_device_tables(dev, &a.tw);
    if (st != W1_OK) return st;
    PdScratch sc;
    st = pd_scratch(sc, a, nx, ny, h);
    if (st != W1_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    W1_CK(cudaMemcpyAsync(sc.w, r, (size_t)nx * ny * sizeof(float), cudaMemcpyDeviceToDevice, s));
    // the potential kernel with phi = 0 would add a divergence: run the bare solve
    W1_CK(launch_pd_poisson(a, psi, 1.f, s));
    W1_CK(cudaStreamSynchronize(s));
    return W1_OK;
}

extern "C" w1_status w1_pdhg_steps(int nx, int ny, double h, int norm, float mu, float tau, const float* rho,
                                   float* m1, float* m2, float* phi1, float* phi2, float* phibar1, float* phibar2,
                                   long long iters, void* stream, double* g_last)
{
    if (!rho || !m1 || !m2 || !phi1 || !phi2 || !phibar1 || !phibar2 || !(h > 0.0) || iters < 0)
        return fail(W1_ERR_INVALID_ARG, "bad arguments to w1_pdhg_steps");
    if (norm != W1_NORM_L1 && norm != W1_NORM_L2 && norm != W1_NORM_LINF) return fail(W1_ERR_INVALID_ARG, "norm must be 1, 2 or 3");
    if (!pd_level_ok(nx, ny)) return fail(W1_ERR_UNSUPPORTED, "nx and ny must be powers of two in [2, 1024]");
    int dev = 0;
    W1_CK(cudaGetDevice(&dev));
    w1_status st = prepare_device(dev);
    if (st != W1_OK) return st;
    PdArgs a{};
    st = pd_device_tables(dev, &a.tw);
    if (st != W1_OK) return st;
    PdScratch sc;
    st = pd_scratch(sc, a, nx, ny, h);
    if (st != W1_OK) return st;
    a.mu = mu;
    a.tau = tau;
    a.rho = rho;
    a.m1 = m1;
    a.m2 = m2;
    a.f1 = phi1;
    a.f2 = phi2;
    a.g1 = phibar1;
    a.g2 = phibar2;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (long long k = 0; k < iters; ++k) W1_CK(launch_pd_step(norm, k + 1 == iters, a, s));
    double g = 0.0;
    if (iters > 0) W1_CK(cudaMemcpyAsync(&g, sc.g, sizeof(double), cudaMemcpyDeviceToHost, s));
    W1_CK(cudaStreamSynchronize(s));
    if (g_last) *g_last = g;
    return W1_OK;
}

extern "C" w1_status w1_cp_steps(int nx, int ny, double h, int norm, float mu, float tau, const float* rho,
                                 float* m1, float* m2, float* phi, long long iters, int path, void* stream,
                                 double* fpr_last)
{
    return w1_cp_steps_ex(nx, ny, h, norm, mu, tau, rho, m1, m2, phi, iters, path, 0, stream, fpr_last);
}

extern "C" w1_status w1_cp_steps_ex(int nx, int ny, double h, int norm, float mu, float tau, const float* rho,
                                    float* m1, float* m2, float* phi, long long iters, int path, int cluster,
                                    void* stream, double* fpr_last)
{
    if (nx < 1 || ny < 1 || !(h > 0.0) || !rho || !m1 || !m2 || !phi || iters < 0)
        return fail(W1_ERR_INVALID_ARG, "bad arguments to w1_cp_steps");
    if (norm != W1_NORM_L1 && norm != W1_NORM_L2 && norm != W1_NORM_LINF) return fail(W1_ERR_INVALID_ARG, "norm must be 1, 2 or 3");
    if ((reinterpret_cast<uintptr_t>(rho) | reinterpret_cast<uintptr_t>(m1) | reinterpret_cast<uintptr_t>(m2) |
         reinterpret_cast<uintptr_t>(phi)) % 16 != 0)
        return fail(W1_ERR_INVALID_ARG, "planes must be 16-byte aligned");
    int dev = 0;
    W1_CK(cudaGetDevice(&dev));
    w1_status st = prepare_device(dev);
    if (st != W1_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (iters == 0) {
        if (fpr_last) *fpr_last = 0.0;
        return W1_OK;
    }
    double* dfpr = nullptr;
    W1_CK(cudaMalloc(&dfpr, sizeof(double)));
    IterArgs it{};
    it.nx = nx;
    it.ny = ny;
    it.mu = mu;
    it.tau = tau;
    it.ih = (float)(1.0 / h);
    it.h = h;
    it.tol = 0.0;
    it.cap = iters;
    it.K = 2;
    it.fixed = 1;
    it.level = 0;
    it.budget_ns = 600ull * 1000000000ull;
    it.stride = (long long)nx * ny;
    it.ctl = nullptr;
    it.fpr_out = dfpr;
    w1_status ret = W1_OK;
    if (path == 1) {
        const int c = cluster > 0 ? cluster : resident_cluster_for(nx, ny);
        if (c == 0 || resident_cluster_ok(norm, c, nx, ny) <= 0) {
            cudaFree(dfpr);
            return fail(W1_ERR_UNSUPPORTED, "this grid does not fit the resident path with this cluster size");
        }
        ResArgs a{};
        a.m1 = m1;
        a.m2 = m2;
        a.phi = phi;
        a.rho = rho;
        a.pairs = 1;
        a.it = it;
        cudaError_t e = launch_resident(norm, c, a, s);
        if (e != cudaSuccess) ret = fail(W1_ERR_CUDA, std::string("resident launch: ") + cudaGetErrorString(e));
    } else {
        // path 3: `cluster` k >= 1 selects tile variant k - 1 (as w1_options.tile); 0 the first
        const int tile = (path == 3 && cluster > 0) ? cluster - 1 : 0;
        if (path == 3 && (cluster < 0 || cluster > W1_TILE_VARIANTS)) {
            cudaFree(dfpr);
            return fail(W1_ERR_INVALID_ARG, "tile variant out of range");
        }
        if (path == 3 && (nx % 4 != 0 || iters % tblock_depth(tile) != 0)) {
            cudaFree(dfpr);
            return fail(W1_ERR_UNSUPPORTED, "temporal blocking needs nx % 4 == 0 and iters a multiple of its depth");
        }
        const size_t n = (size_t)nx * ny;
        const int rows = stream_rows_auto(nx, ny, 1);
        const long long launches = path == 3 ? iters / tblock_depth(tile) : iters;
        size_t pd = step_part_doubles(nx, ny, rows, 1);
        if (tblock_part_doubles(nx, ny, 1) > pd) pd = tblock_part_doubles(nx, ny, 1);
        float* buf = nullptr;
        double* part = nullptr;
        Ctl* ctl = nullptr;
        cudaError_t e = cudaMalloc(&buf, 3 * n * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&part, pd * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&ctl, sizeof(Ctl));
        if (e == cudaSuccess) e = cudaMemsetAsync(ctl, 0, sizeof(Ctl), s);
        float* A[3] = {m1, m2, phi};
        float* B[3] = {buf, buf + n, buf + 2 * n};
        for (long long k = 0; k < launches && e == cudaSuccess; ++k) {
            float** src = (k & 1) ? B : A;
            float** dst = (k & 1) ? A : B;
            StepArgs a{};
            a.m1 = src[0];
            a.m2 = src[1];
            a.phi = src[2];
            a.rho = rho;
            a.m1o = dst[0];
            a.m2o = dst[1];
            a.phio = dst[2];
            a.rows = rows;
            a.pairs = 1;
            a.it = it;
            a.it.ctl = ctl;
            a.part = part;
            a.use_cond = 0;
            a.tile = tile;
            e = path == 3 ? launch_tblock(norm, k == launches - 1, a, s) : launch_step(norm, k == launches - 1, a, s);
        }
        if (e == cudaSuccess && (launches & 1)) {
            for (int c = 0; c < 3 && e == cudaSuccess; ++c)
                e = cudaMemcpyAsync(A[c], B[c], n * sizeof(float), cudaMemcpyDeviceToDevice, s);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) ret = fail(W1_ERR_CUDA, std::string("streaming steps: ") + cudaGetErrorString(e));
        cudaFree(buf);
        cudaFree(part);
        cudaFree(ctl);
    }
    if (ret == W1_OK) {
        double v = 0.0;
        cudaError_t e = cudaMemcpyAsync(&v, dfpr, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) ret = fail(W1_ERR_CUDA, std::string("fpr readback: ") + cudaGetErrorString(e));
        if (fpr_last) *fpr_last = v;
    }
    cudaFree(dfpr);
    cudaGetLastError();
    return ret;
}

extern "C" w1_status w1_restrict(int nx, int ny, const float* fine, float* coarse, void* stream)
{
    if (nx < 2 || ny < 2 || (nx & 1) || (ny & 1) || !fine || !coarse)
        return fail(W1_ERR_INVALID_ARG, "w1_restrict needs even nx, ny >= 2");
    W1_CK(launch_restrict(fine, nx, ny, coarse, 1, nullptr, static_cast<cudaStream_t>(stream)));
    return W1_OK;
}

extern "C" w1_status w1_prolong(int ncx, int ncy, const float* m1c, const float* m2c, const float* phic, float* m1f,
                                float* m2f, float* phif, void* stream)
{
    if (ncx < 1 || ncy < 1 || !m1c || !m2c || !phic || !m1f || !m2f || !phif)
        return fail(W1_ERR_INVALID_ARG, "bad arguments to w1_prolong");
    W1_CK(launch_prolong(ncx, ncy, m1c, m2c, phic, m1f, m2f, phif, 1, nullptr, static_cast<cudaStream_t>(stream)));
    return W1_OK;
}

extern "C" w1_status w1_state_stats(int nx, int ny, double h, int norm, const float* rho, const float* m1,
                                    const float* m2, const float* phi, void* stream, w1_stats* out)
{
    if (nx < 1 || ny < 1 || !(h > 0.0) || !rho || !m1 || !m2 || !phi || !out)
        return fail(W1_ERR_INVALID_ARG, "bad arguments to w1_state_stats");
    if (norm != W1_NORM_L1 && norm != W1_NORM_L2 && norm != W1_NORM_LINF) return fail(W1_ERR_INVALID_ARG, "norm must be 1, 2 or 3");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t n = (size_t)nx * ny;
    double *q = nullptr, *part = nullptr;
    Ctl* ctl = nullptr;
    cudaError_t e = cudaMalloc(&q, 2 * n * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&part, final_part_doubles(1) * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&ctl, sizeof(Ctl));
    if (e == cudaSuccess) e = cudaMemsetAsync(ctl, 0, sizeof(Ctl), s);
    if (e == cudaSuccess) e = launch_final(norm, m1, m2, phi, rho, nx, ny, h, q, part, ctl, 1, s);
    Ctl c{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&c, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(q);
    cudaFree(part);
    cudaFree(ctl);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(W1_ERR_CUDA, std::string("w1_state_stats: ") + cudaGetErrorString(e));
    }
    std::memset(out, 0, sizeof(*out));
    out->w1 = c.saddle;
    out->primal = c.f;
    out->saddle = c.saddle;
    out->dual = c.dual;
    out->lb = c.lb;
    out->ub = c.ub;
    out->route = c.route;
    out->res_l1 = c.res_l1;
    out->rho_l1 = c.rho_l1;
    out->gmax = c.gmax;
    return W1_OK;
}
