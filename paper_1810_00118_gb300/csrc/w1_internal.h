// w1_internal.h -- declarations shared by the kernels and the host driver of the
// GB300 W1 library (not part of the public ABI; include/w1.h is).
//
// Batching: a plan holds `B` pairs of the same grid.  Every plane of level l is
// stored as B consecutive [ny_l][nx_l] planes (pair stride n_l = nx_l * ny_l),
// and every kernel takes the pair from its grid (blockIdx.z, blockIdx.y, or the
// cluster index), so one launch advances all pairs.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdio>
#include <stdint.h>

#include "../../include/w1.h"

namespace w1 {

// NVTX range on the host timeline (a no-op unless a profiler is attached):
// plan solves, levels of eager and 3-D solves, server requests, autotuning.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    template <class... A>
    NvtxRange(const char* fmt, A... a)
    {
        char buf[96];
        std::snprintf(buf, sizeof(buf), fmt, a...);
        nvtxRangePushA(buf);
    }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Per-pair device control block: reduction counter, flags, per-level iteration
// counts and residuals, and the final statistics.
struct Ctl {
    unsigned int counter;  // last-block counter of this pair's grid reductions (reset by the last block)
    int error;             // 0 ok, 1 rejected input (mass or non-finite), 2 unused batch slot
    int timeout;           // 1: a level hit the wall-clock guard
    int active;            // streaming level: 1 while this pair still iterates
    double mass0, mass1, mean;
    long long iters[W1_MAX_LEVELS];
    double fpr[W1_MAX_LEVELS];
    int conv[W1_MAX_LEVELS];
    unsigned long long t_start[W1_MAX_LEVELS];
    // final statistics of the returned finest state (saddle: the Lagrangian of
    // eq. minmax_cp at the state)
    double f, dual, res_l1, rho_l1, gmax, route, lb, ub, saddle;
};

// Iteration arguments shared by both level paths.
struct IterArgs {
    int nx, ny;
    float mu, tau, ih;  // step sizes and 1/h, as the FP32 iteration uses them
    double h;           // spacing for the FP64 residual sums
    double tol;         // eps_l
    long long cap;      // max steps (or the exact step count when fixed)
    int K;              // steps between stop tests
    int fixed;          // 1: take exactly `cap` steps, form R^k of the last one
    int level;
    unsigned long long budget_ns;
    long long stride;      // elements between consecutive pairs' planes
    Ctl* ctl;              // per-pair control blocks (may be null for building blocks)
    double* fpr_out;       // optional (device, per pair): R^k of the last tested step
    long long* iters_out;  // optional (device, per pair)
};

// Streaming (global memory) one-step kernel arguments; pointers are pair 0's planes.
struct StepArgs {
    const float* m1;
    const float* m2;
    const float* phi;
    const float* rho;
    float* m1o;
    float* m2o;
    float* phio;
    int rows;  // rows marched per thread
    int pairs;
    IterArgs it;
    double* part;  // per-pair, per-block partials (check step)
    int use_cond;  // graph mode: keep per-pair active flags and counts
    int tile;      // temporally blocked launches: the tile variant (index into the tile table)
};

// Shared-memory resident level solver arguments (state in place).
struct ResArgs {
    float* m1;
    float* m2;
    float* phi;
    const float* rho;
    int pairs;
    IterArgs it;
    // fault injection for tests of the bounded halo waits: CTA (drop_rank - 1)
    // of every cluster skips its halo pushes (0: none; the host sets it from
    // the W1_FAULT_HALO_RANK environment variable when a plan is built)
    int drop_rank;
};

// W1_FAULT_HALO_RANK=r makes CTA r of every on-chip cluster level skip its halo
// pushes, so that its neighbours' bounded waits run out and the level ends with
// a timeout status (tests of that path only); returns r + 1, or 0 when unset.
int fault_halo_rank();

// Kernel launchers (w1_kernels.cu).  All enqueue on `s` and return the launch status.
// prep: rho = rho0 - rho1 per pair, mass check, exact zero mean; pairs >= nbatch are
// marked unused.  r0, r1 and rho have pair stride n.
cudaError_t launch_prep(const float* r0, const float* r1, long long n, int nbatch, int pairs, double h, Ctl* ctl,
                        double* part, float* rho, cudaStream_t s);
size_t prep_part_doubles(int pairs);
cudaError_t launch_restrict(const float* fine, int nx, int ny, float* coarse, int pairs, const Ctl* ctl,
                            cudaStream_t s);
cudaError_t launch_prolong(int ncx, int ncy, const float* m1c, const float* m2c, const float* phic, float* m1f,
                           float* m2f, float* phif, int pairs, const Ctl* ctl, cudaStream_t s);
cudaError_t launch_level_begin(Ctl* ctl, int level, int pairs, cudaStream_t s);
// Streaming step; check selects the variant that forms R^k and tests it.
cudaError_t launch_step(int norm, bool check, const StepArgs& a, cudaStream_t s);
// Temporally blocked streaming steps: tblock_depth(a.tile) steps per launch
// on tiles of the variant a.tile (the last step forms R^k when check is set);
// same arguments as launch_step.  Partial sums: at most tblock_part_doubles
// (the largest over the variants).
cudaError_t launch_tblock(int norm, bool check, const StepArgs& a, cudaStream_t s);
int tblock_depth(int tile = 0);
dim3 tblock_grid(int nx, int ny, int pairs, int tile = 0);
size_t tblock_part_doubles(int nx, int ny, int pairs);
// After a check step in graph mode: continue the WHILE node while any pair is active.
cudaError_t launch_decide(const Ctl* ctl, int pairs, cudaGraphConditionalHandle cond, cudaStream_t s);
int stream_rows_auto(int nx, int ny, int pairs);
dim3 stream_grid(int nx, int ny, int rows, int pairs);
size_t step_part_doubles(int nx, int ny, int rows, int pairs);
// Resident level solve with a cluster of `cluster` CTAs per pair.
cudaError_t launch_resident(int norm, int cluster, const ResArgs& a, cudaStream_t s);
int resident_max_nodes();
// Whether a level of nx x ny fits on chip in a cluster of `cluster` CTAs (bands of
// whole rows: at most 4096 nodes per CTA, or 16384 with 16 CTAs and nx % 4 == 0).
bool resident_fits(int nx, int ny, int cluster);
int resident_cluster_for(int nx, int ny);
cudaError_t resident_prepare(int device);
// Active clusters the device can hold for this configuration (0: cannot launch).
int resident_cluster_ok(int norm, int cluster, int nx, int ny);
// Mixed-size batches: one persistent launch runs the whole cascade of
// Algorithm 3 (prolongation and every level's solve) for pairs of several grid
// sizes, one CTA per pair; CTAs take pairs from a shared counter, largest grids
// first.  Restriction, prep and the final statistics stay batched launches per
// size class.
struct CascadeLevel {
    int nx, ny;
    // how a cluster of CASCADE_CLUSTER CTAs solves the level of a pair of a
    // cluster class: CASCADE_SPLIT4 / CASCADE_SPLITW in row bands over the
    // cluster (four-nodes-per-thread or wide layout), CASCADE_ONE4 /
    // CASCADE_ONEW on CTA 0 alone; unused for single-CTA classes
    int mode;
    float mu, tau, ih;
    double h, tol;
    float* rho;  // pair 0's planes of this level; pair stride nx * ny
    float* m1;
    float* m2;
    float* phi;
};
struct CascadeClass {
    int levels, count;
    // levels 0 .. split - 1 (at most CASCADE_COARSE_NODES nodes each) run in the
    // coarse launch, levels split .. levels - 1 in the persistent launch
    int split;
    Ctl* ctl;  // per-pair control blocks of the class
    CascadeLevel lv[W1_MAX_LEVELS];
};
struct CascadeArgs {
    const CascadeClass* cls;  // device array: classes whose pairs one CTA solves
    int n_classes;
    int total;            // pairs over all classes
    unsigned int* next;   // work counter, zero before the launch
    long long cap;        // per-level step cap
    int K;                // steps between stop tests
    unsigned long long budget_ns;
    // cluster launch only: classes whose pairs a cluster of CASCADE_CLUSTER
    // CTAs solves (taken first), and their work counter
    const CascadeClass* big;
    int n_big;
    int total_big;
    unsigned int* next_big;
};
static constexpr int CASCADE_CLUSTER = 4;
// Levels of at most this many nodes run in the coarse launch (CTAs of
// CASCADE_COARSE_THREADS threads, several per SM) before the persistent launch.
static constexpr int CASCADE_COARSE_NODES = 1024;
static constexpr int CASCADE_COARSE_THREADS = 256;
enum { CASCADE_SPLIT4 = 1, CASCADE_SPLITW = 2, CASCADE_ONE4 = 3, CASCADE_ONEW = 4 };
// Which single-CTA layouts hold an nx x ny level (nx % 4 == 0): bit 0 four
// nodes per thread (at most 4096 nodes), bit 1 wide (at most 16384 nodes, a
// multiple of 128).  A persistent launch with wide = false runs only levels of
// the first kind; with wide = true, larger levels on the wide layout.
int cascade_level_fits(int nx, int ny);
// CTAs of the persistent launch that fit the device at once.
int cascade_ctas(int norm, bool wide);
cudaError_t launch_cascade(int norm, bool wide, const CascadeArgs& a, int ctas, cudaStream_t s);
// How a cluster of CASCADE_CLUSTER CTAs solves an nx x ny level (a CASCADE_*
// mode), or 0 when it cannot.
int cascade_level_mode_cluster(int nx, int ny);
// Clusters of the cluster persistent launch that fit the device at once.
int cascade_clusters(int norm);
// The persistent launch with clusters of CASCADE_CLUSTER CTAs: each cluster
// takes pairs of a.big together, then each of its CTAs pairs of a.cls alone.
cudaError_t launch_cascade_cluster(int norm, const CascadeArgs& a, int clusters, cudaStream_t s);
// The coarse launch: pairs of a.cls (every persistent class), levels 0 ..
// split - 1, one pair per CTA of CASCADE_COARSE_THREADS threads; CTAs resident
// at once from cascade_coarse_ctas.
int cascade_coarse_ctas(int norm);
cudaError_t launch_cascade_coarse(int norm, const CascadeArgs& a, int ctas, cudaStream_t s);
// Prox-PDHG (Algorithm 2 on one level; Algorithm 4 through the plan).  Every
// plane holds the batch's pairs back to back (pair stride nx * ny).
struct PdArgs {
    int nx, ny, pairs;
    float mu, tau, ih;
    double h, tol;
    long long stride;
    const float* rho;
    float* m1;
    float* m2;
    float* f1;  // phi (the dual vector field)
    float* f2;
    float* g1;  // phibar
    float* g2;
    float* w;  // residual / potential of the Poisson solve
    float* t;  // transposed scratch
    const float2* tw;  // e^{-2 pi i k / 4096}, k < 4096
    const float* lamx;  // (2 - 2 cos(pi k / nx)) / h^2
    const float* lamy;
    Ctl* ctl;          // may be null (building blocks)
    double* part;      // per-pair, per-block partials of the test step
    double* g_out;     // optional (device, per pair): G^k of the last test step
    int use_cond;      // keep per-pair active flags and counts (level loops)
    int level, K;
    long long cap;
    unsigned long long budget_ns;
};
bool pd_level_ok(int nx, int ny);  // both sides powers of two in [2, 1024]
size_t pd_twiddle_count();
void pd_twiddles(float2* host);                 // pd_twiddle_count() entries
void pd_eigen(int n, double h, float* host);    // n entries
size_t pd_part_doubles(int nx, int ny, int pairs);
cudaError_t pd_prepare();
// One step of eq. pdhg (5 launches); check forms G^k and, with use_cond, the stop decision.
cudaError_t launch_pd_step(int norm, bool check, const PdArgs& a, cudaStream_t s);
// The Neumann Poisson solve on a.w (in place, or scale * psi into dst).
cudaError_t launch_pd_poisson(const PdArgs& a, float* dst, float scale, cudaStream_t s);
// phi_out = the Kantorovich potential recovered from phi (Appendix B), sign of Algorithm 1's.
cudaError_t launch_pd_potential(const PdArgs& a, float* phi_out, cudaStream_t s);
// Final statistics of a state into ctl (q: FP64 scratch of 2 * nx * ny per pair).
// The first kernel runs FIN_BLOCKS_PER_PAIR blocks per pair, each leaving
// FIN_PART_PER_BLOCK doubles of partial sums: final_part_doubles(pairs) =
// FIN_BLOCKS_PER_PAIR * FIN_PART_PER_BLOCK * pairs.
static constexpr int FIN_BLOCKS_PER_PAIR = 64;
static constexpr int FIN_PART_PER_BLOCK = 13;  // six compensated sums (s, c) and a maximum
cudaError_t launch_final(int norm, const float* m1, const float* m2, const float* phi, const float* rho, int nx,
                         int ny, double h, double* q, double* part, Ctl* ctl, int pairs, cudaStream_t s);
size_t final_part_doubles(int pairs);

}  // namespace w1
