/*
 * w1.h -- C ABI of the GB300 multilevel primal-dual Wasserstein-1 solver.
 *
 * Method: Liu, Yin, Li, Chow, "Multilevel Optimal Transport: a Fast
 * Approximation of Wasserstein-1 distances" (arXiv 1810.00118).
 *   - The problem is the discrete Beckmann (minimal flux) form of W1,
 *       min_m  sum_x ||m(x)||_p h^2   s.t.  div^h m = rho0 - rho1,
 *     zero-flux boundary, on a uniform 2-D grid (Sec. 2.2, eq. opt_flux_dis).
 *   - Each level runs Algorithm 1, the primal-dual iteration of eq. primaldual:
 *       m   <- prox_{mu||.||_p}(m + mu grad phi)      (shrink toward m + mu grad phi)
 *       phi <- phi + tau (div(2 m_new - m_old) - rho) (dual ascent, extrapolated residual)
 *   - Algorithm 3 solves coarse to fine: densities are restricted by 2x2 block
 *     means, and (m, phi) of level l-1 are interpolated (Sec. 3.3) to start level l.
 *
 * Grid and layout (all entry points):
 *   - nx * ny nodes at pixel centres, spacing h; node (i, j), i along x.
 *   - Every plane is float32, dense, row-major [ny][nx] (index j*nx + i).
 *   - A flux is two planes, m1 (x-edges (i,j)->(i+1,j)) then m2 (y-edges
 *     (i,j)->(i,j+1)); m1[j][nx-1] and m2[ny-1][i] are always 0.
 *   - Level l of L has (nx, ny) / 2^(L-l) nodes and spacing h * 2^(L-l);
 *     nx and ny must be divisible by 2^(L-1).
 *
 * Stopping rule (Algorithm 1 with eq. pd_stop): after every K-th step the
 * fixed-point residual R^k of that step is formed on the device (FP64 sums);
 * level l stops when R^k < eps_l, eps_l = tol * (h_l / h)^alpha
 * (eq. tol_formula_propose; alpha = -1 and tol from eq. stop_tol are the
 * paper's choices).  Iteration counts are therefore multiples of K.
 *
 * Errors: no entry point aborts; every one returns a w1_status.  The text of
 * the last error of the calling thread is available from w1_last_error().
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream).  Work is enqueued on it in order; calls that return host values
 * synchronise with it before returning.
 */
#ifndef W1_H_
#define W1_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define W1_MAX_LEVELS 16
#define W1_TILE_VARIANTS 5 /* tile shapes of the temporally blocked streaming kernel */
#define W1_TUNE_MAX_CANDIDATES 16 /* configurations w1_autotune_level reports at most */

typedef enum {
    W1_NORM_L1 = 1,  /* p = 1, anisotropic: ||m(x)|| = |m1| + |m2|, componentwise shrink */
    W1_NORM_L2 = 2,  /* p = 2, isotropic:  ||m(x)|| = sqrt(m1^2 + m2^2), vector shrink  */
    W1_NORM_LINF = 3 /* p = infinity: ||m(x)|| = max(|m1|, |m2|); shrink by the Moreau
                        decomposition v - mu Proj_{l1 ball}(v / mu) (Sec. 4)          */
} w1_norm;

typedef enum {
    W1_OK = 0,
    W1_ERR_INVALID_ARG = 1,   /* a NULL pointer, a non-positive size, an unknown norm  */
    W1_ERR_SHAPE = 2,         /* nx or ny not divisible by 2^(levels-1), or too many levels */
    W1_ERR_MASS = 3,          /* |M0 - M1| > 1e-6 max(|M0|,|M1|) or a non-finite input   */
    W1_ERR_NOMEM = 4,         /* device or pinned host allocation failed                 */
    W1_ERR_CUDA = 5,          /* a CUDA call failed (message in w1_last_error)           */
    W1_ERR_NOT_CONVERGED = 6, /* a level hit max_iters; dist and stats are still written */
    W1_ERR_TIMEOUT = 7,       /* a level hit the device wall-clock guard; ditto          */
    W1_PENDING = 8,           /* w1_poll: the request has not finished                   */
    W1_ERR_BUDGET = 9,        /* w1_submit: request larger than the server's HBM budget  */
    W1_ERR_UNSUPPORTED = 10   /* a feature this build or device does not provide         */
} w1_status;

/* Plan options; w1_default_options() fills the defaults given here. */
typedef struct {
    int check_every;       /* K: steps between stop tests, a multiple of 8; 0 (default): 32
                              for Algorithm 3 (64 with schedule = 1 for p = 1, 2), 8 for
                              Algorithm 4                                                    */
    long long max_iters;   /* cap on steps per level (default 1000000)                        */
    double theta;          /* mu = tau = theta / ||A_h||, ||A_h|| <= 2 sqrt(2) / h (Sec. 4);
                              0.5 is the paper's choice (default), 1.0 its footnote's         */
    double alpha;          /* eps_l = tol * (h_l / h)^alpha (default -1)                      */
    double time_budget_s;  /* device wall-clock guard per level (default 60 s)               */
    int path;              /* 0 automatic; 1 shared-memory resident; 2 streaming, one step per
                              launch; 3 streaming with temporal blocking (4 steps per launch,
                              needs nx % 4 == 0); automatic = 1 where a level fits on chip,
                              else 3 where possible, else 2                                 */
    int rows_per_thread;   /* streaming kernel: rows marched per thread (0 = automatic)       */
    int eager;             /* 1: launch the level kernels directly and test convergence of
                              streaming levels on the host (for profilers that do not follow
                              conditional graph nodes); 0: one CUDA graph (default)           */
    int tune;              /* 0: fixed rules pick each level's kernel; 1: the autotuner picks
                              the fastest for one pair (latency); 2: the fastest for the
                              plan's batch advancing together (throughput); 3: the least
                              SM-time per step (many independent solves sharing the GPU) */
    int algorithm;         /* 3 (default, 0 too): Algorithm 3, Chambolle-Pock on every level
                              (eq. primaldual, stop R^k < eps_l); 4: Algorithm 4, prox-PDHG
                              (eq. pdhg: projection onto div m = rho by a DCT Poisson solve,
                              stop G^k < eps_l of eq. pdhg_stop; mu = tau = theta, the paper's
                              1/2; tol <= 0 gives eq. stop_tol for Alg. 4); level sides must
                              be powers of two in [2, 1024]; path and tune do not apply    */
    int tile;              /* tile of the temporally blocked levels (path 3): 0 automatic (the
                              first variant, or the autotuner's pick when tune > 0); k in
                              1..W1_TILE_VARIANTS forces variant k - 1 of
                                64x32 nodes 4 steps, 128x16 4, 32x64 4, 64x32 8, 32x32 8
                              (interior nodes of a tile and steps per launch; check_every
                              must be a multiple of twice the steps)                       */
    double step_ratio;     /* tau / mu of eq. primaldual at a fixed product mu tau = (theta /
                              ||A_h||)^2: mu = theta / ||A_h|| / sqrt(r), tau = theta / ||A_h||
                              * sqrt(r) (default 1: mu = tau, the paper's); 2-D Algorithm 3 */
    int schedule;          /* level tolerances: 0 (default) eps_l = tol (h_l / h)^alpha as given;
                              1 the calibrated schedule for the saddle-value estimate at
                              relative 1e-4: per norm, an eps_L scale (applied to eq. stop_tol
                              when tol <= 0, whose (512 h)^2 factor is then capped at 1 so
                              that grids coarser than 512^2 keep the 512^2 eps_L), an alpha,
                              a theta and a step ratio that replace
                              opt.alpha, opt.theta and opt.step_ratio, measured on
                              the 512^2 ellipse-texture workload against converged W1 (the
                              fastest setting whose worst error over the calibration pairs was
                              at most 2.5e-5; w1_calibrated_schedule reports the values);
                              p = infinity and 3-D solves keep the paper's values            */
    int estimate;          /* which value dist and w1_stats.w1 report:
                              0 (default): the saddle value, the Lagrangian of eq. minmax_cp
                                L(m, phi) = f(m) + <phi, div m - rho>_h at the returned pair;
                                it corrects f(m) to first order for the constraint residual
                                div m - rho that the stopped iteration leaves;
                              1: the primal objective f(m) of the returned flux (the value
                                Sec. 5 prints as the approximation, f(m^K));
                              both are also in w1_stats.saddle and w1_stats.primal          */
} w1_options;

/* What a solve reports.  Values are FP64 compensated sums (TwoSum error terms
 * carried beside every running sum) of per-node terms of the FP32 state. */
typedef struct {
    int levels;
    int nx[W1_MAX_LEVELS];          /* level sizes, coarsest first */
    int ny[W1_MAX_LEVELS];
    long long iters[W1_MAX_LEVELS]; /* steps taken on each level */
    double fpr[W1_MAX_LEVELS];      /* R^k at the last stop test of each level */
    double tol[W1_MAX_LEVELS];      /* eps_l of each level */
    int path[W1_MAX_LEVELS];        /* 1 resident (cluster size in cluster[]), 2 streaming, 3 blocked */
    int cluster[W1_MAX_LEVELS];     /* path 1: CTAs per pair; path 3: tile variant + 1 (w1_options.tile) */
    double w1;       /* the W1 estimate chosen by w1_options.estimate (default: saddle) */
    double dual;     /* -<phi, rho>_h of the returned potential */
    double lb;       /* certified lower bound on the discrete W1: dual / max(1, gmax) */
    double ub;       /* certified upper bound: primal + route */
    double route;    /* cost of an explicit flux carrying the residual rho - div m */
    double res_l1;   /* sum |rho - div m| h^2 */
    double rho_l1;   /* sum |rho| h^2 */
    double gmax;     /* max over nodes of ||grad phi(x)||_q (q dual to p: inf, 2, 1) */
    double mass0;    /* sum rho0 h^2 */
    double mass1;    /* sum rho1 h^2 */
    double mass_shift; /* mean of rho0 - rho1 removed so that the constraint is solvable */
    int converged;   /* 1 when every level met its tolerance */
    double primal;   /* f(m) = sum ||m(x)||_p h^2 of the returned flux (eq. opt_flux_dis) */
    double saddle;   /* L(m, phi) = f(m) + <phi, div m - rho>_h (eq. minmax_cp)           */
} w1_stats;

typedef struct w1_plan w1_plan;

/* Fills *opt with the defaults documented in w1_options. */
void w1_default_options(w1_options* opt);
/* The calibrated schedule of w1_options.schedule = 1 for a norm: the factor on
 * eq. stop_tol's eps_L, the alpha of eq. tol_formula_propose, the step-size
 * factor theta and the step ratio tau / mu (host only, needs no device).  The paper has no counterpart: the
 * values come from measurement against converged W1 (see w1_options.schedule). */
w1_status w1_calibrated_schedule(int norm, double* tol_scale, double* alpha, double* theta, double* step_ratio);

/*
 * Creates a plan for nx x ny grids (Algorithm 3 input, Sec. 3.2).
 *   h      : finest spacing; <= 0 means 1 / max(nx, ny).
 *   levels : L; <= 0 means the paper's L = log2(1/h) - 3 (Sec. 5.3), reduced
 *            until nx and ny are divisible by 2^(L-1) and the coarsest side >= 2.
 *   norm   : W1_NORM_L1, W1_NORM_L2 or W1_NORM_LINF.
 *   tol    : eps_L of the finest level; <= 0 means eq. stop_tol for Alg. 3,
 *            eps_L = 1e-6/128 * (512 h)^2.
 * The plan owns its device workspace (allocated on the current device) unless
 * w1_plan_set_workspace() hands it one.  Returns W1_ERR_SHAPE on bad sizes.
 */
w1_status w1_plan_create(int nx, int ny, double h, int levels, int norm, double tol, w1_plan** out);
w1_status w1_plan_create_ex(int nx, int ny, double h, int levels, int norm, double tol, const w1_options* opt,
                            w1_plan** out);
w1_status w1_plan_destroy(w1_plan* plan);

/*
 * A plan for batches of up to max_batch pairs of the same grid (every kernel
 * launch advances all pairs of the batch).  Arguments
 * as w1_plan_create_ex.  Device memory grows linearly with max_batch.
 */
w1_status w1_plan_create_batch(int nx, int ny, double h, int levels, int norm, double tol, int max_batch,
                               const w1_options* opt, w1_plan** out);
int w1_plan_max_batch(const w1_plan* plan);

/* Bytes of device workspace the plan needs (levels' state, reductions). */
size_t w1_plan_workspace_bytes(const w1_plan* plan);
/* Use caller-owned device memory (>= w1_plan_workspace_bytes, 256-byte aligned)
 * instead of the plan's own; the caller keeps it alive until the plan dies. */
w1_status w1_plan_set_workspace(w1_plan* plan, void* device_ptr, size_t bytes);

/*
 * One W1 solve (Algorithm 3), enqueued on `stream`.
 *   rho0, rho1 : device, [ny][nx] float32 densities, caller-owned, read only.
 *   dist       : host; receives the W1 estimate (w1_options.estimate; blocks until the stream
 *                reaches the end of the solve).
 *   flux       : device [2][ny][nx] float32 (m1 then m2) or NULL.
 *   stats      : host or NULL.
 * Returns W1_OK, W1_ERR_MASS (nothing solved), W1_ERR_NOT_CONVERGED or
 * W1_ERR_TIMEOUT (dist and stats still written), or an error.
 */
w1_status w1_solve(w1_plan* plan, const float* rho0, const float* rho1, void* stream, double* dist, float* flux,
                   w1_stats* stats);

/*
 * Solves `batch` pairs (1 <= batch <= max_batch) in one pass of Algorithm 3.
 *   rho0, rho1 : device, [batch][ny][nx] float32.
 *   dist       : host [batch].  flux: device [batch][2][ny][nx] or NULL.
 *   stats      : host [batch] or NULL.  status: host [batch] or NULL, each
 *                pair's own status (W1_OK, W1_ERR_MASS, W1_ERR_NOT_CONVERGED,
 *                W1_ERR_TIMEOUT).
 * Pairs are independent: each stops on its own test, and a rejected pair does
 * not affect the others.  Returns W1_OK when every pair is W1_OK, else the
 * first pair's non-OK status (dist of a rejected pair is NaN).
 */
w1_status w1_solve_batch(w1_plan* plan, int batch, const float* rho0, const float* rho1, void* stream, double* dist,
                         float* flux, w1_stats* stats, int* status);
/*
 * Asynchronous solve: enqueues everything w1_solve_batch does on `stream` and
 * returns without waiting.  Once the stream has passed the enqueued work
 * (cudaStreamSynchronize, an event, a host callback), w1_plan_results() gives
 * dist, stats and per-pair status exactly as w1_solve_batch would.  A plan
 * holds the results of its last enqueued solve only, and must not have two
 * solves in flight at once (use one plan per stream for concurrent solves;
 * their work overlaps on the device).  rho0/rho1/flux must stay valid until
 * the stream has passed the solve.
 */
w1_status w1_solve_async(w1_plan* plan, int batch, const float* rho0, const float* rho1, void* stream, float* flux);
w1_status w1_plan_results(w1_plan* plan, double* dist, w1_stats* stats, int* status);

/* w1_solve_batch for host (pageable or pinned) densities and flux; the copies
 * to and from the device are part of the call.  The call waits for its solve
 * asleep (an event with blocking synchronisation) rather than spinning, so that
 * many host threads calling it at once do not take each other's cores. */
w1_status w1_solve_batch_host(w1_plan* plan, int batch, const float* rho0, const float* rho1, void* stream,
                              double* dist, float* flux, w1_stats* stats, int* status);

/* Same as w1_solve, for densities and flux in (pageable or pinned) host
 * memory: the copies to and from the device are part of the call (and the
 * wait is asleep, as w1_solve_batch_host's). */
w1_status w1_solve_host(w1_plan* plan, const float* rho0, const float* rho1, void* stream, double* dist,
                        float* flux, w1_stats* stats);

/* Final potential phi of the last solve, device [batch][ny][nx] float32 (the
 * Kantorovich potential of Algorithm 1, Appendix B); enqueued on stream. */
w1_status w1_plan_potential(w1_plan* plan, float* phi, void* stream);

/* ------------------------------------------------------------------------- */
/* Mixed-size batches                                                        */
/* ------------------------------------------------------------------------- */

typedef struct w1_mixed w1_mixed;

/*
 * A batch of pairs of several grid sizes, solved together (Algorithm 3 for
 * every pair).  Class c has count[c] pairs of nx[c] x ny[c] (levels and h as
 * w1_plan_create with levels = 0, h = 0).  Classes whose every level fits one
 * CTA (nx % 4 == 0 at every level, at most 16384 nodes) run in ONE persistent
 * launch: each CTA takes a pair, runs all of its levels (interpolation and the
 * level solves) on chip, and takes the next pair, largest grids first.  When a
 * class has a level larger than one CTA holds that four CTAs hold in row bands
 * (each at most 16384 nodes, nx <= 4096), the persistent launch runs in clusters
 * of four CTAs: clusters take those pairs first (their larger levels split over
 * the cluster), then every CTA takes pairs of the other classes alone.  The
 * levels of at most 1024 nodes of every pair run before, in a coarse launch of
 * 256-thread CTAs (several to an SM), one pair per CTA.  Classes that fit
 * neither run as batched plans on streams of their own, overlapping the
 * persistent launch.  opt->path != 0 sends every class to the batched plans.
 * The batch owns its device memory (one arena per class).
 */
w1_status w1_mixed_create(int n_classes, const int* nx, const int* ny, const int* count, int norm, double tol,
                          const w1_options* opt, w1_mixed** out);
w1_status w1_mixed_destroy(w1_mixed* batch);
/* 1 if class cls runs in the persistent launch, 0 if as a batched plan, -1 on bad arguments. */
int w1_mixed_persistent(const w1_mixed* batch, int cls);
/* The persistent launches' sizes (0 where a launch is not used): CTAs of the
 * single-CTA persistent launch (beside the cluster launch, on the SMs no whole
 * cluster uses, when there is one), clusters of the cluster launch, CTAs of the
 * coarse launch.  Any output may be NULL. */
w1_status w1_mixed_launch_info(const w1_mixed* batch, int* ctas, int* clusters, int* coarse_ctas);
/*
 * Enqueues a solve of every pair on `stream` and returns without waiting.
 * rho0[c], rho1[c]: device [count[c]][ny[c]][nx[c]] float32 (host arrays of
 * n_classes device pointers), caller-owned, valid until the stream has passed
 * the solve.  Read the results with w1_mixed_results once the stream is done.
 */
w1_status w1_mixed_solve_async(w1_mixed* batch, const float* const* rho0, const float* const* rho1, void* stream);
/* Results of class cls of the last solve: dist, stats, status as w1_solve_batch (each [count[cls]] or NULL). */
w1_status w1_mixed_results(w1_mixed* batch, int cls, double* dist, w1_stats* stats, int* status);

/* One way to run a level, as measured by the autotuner. */
typedef struct {
    int path;           /* 1 on chip, 2 streaming, 3 streaming with temporal blocking */
    int cluster;        /* CTAs per pair for path 1 */
    int batch;          /* pairs advancing together when it was timed */
    double us_per_step; /* measured time of one step of the whole batch */
    int concurrent;     /* path 1: pairs whose level fits on the GPU at once (CTAs or clusters
                           resident together); streaming: 1 (a launch spans the GPU) */
    int tile;           /* path 3: the tile variant (see w1_options.tile), 0-based */
} w1_level_choice;

/*
 * Times every configuration that can run an nx x ny level (`steps` steps each,
 * synthetic density, CUDA events) and returns the best in `best`.
 * objective 1: fastest for one pair alone (latency); objective 2: fastest for
 * `batch` pairs advancing together as in a batched plan (throughput: a
 * configuration with fewer CTAs per pair can finish a large batch sooner);
 * objective 3: least SM-time per step of one pair (time x SMs it holds: for many
 * independent solves sharing the GPU, as with one plan per stream).  `all` (room
 * for W1_TUNE_MAX_CANDIDATES) receives every
 * measured candidate when not NULL, n_all their number.  Results are cached
 * per device, grid, norm and batch for the process, and in the file named by
 * the environment variable W1_AUTOTUNE_CACHE when it is set.  The choice is
 * the kernel and its cluster size; the tiles of the streaming kernels are
 * fixed at compile time (64 x 32 nodes, 4 steps per launch for path 3).
 * Allocates up to 2 GiB of scratch while it runs.
 */
w1_status w1_autotune_level(int nx, int ny, int norm, int batch, int objective, int steps, w1_level_choice* best,
                            w1_level_choice* all, int* n_all);
const char* w1_autotune_last_error(void);

/* Device bytes a plan with these arguments would allocate (0 on invalid
 * arguments); lets a caller admit work against a memory budget. */
size_t w1_plan_bytes(int nx, int ny, double h, int levels, int norm, double tol, int max_batch,
                     const w1_options* opt);

/* ------------------------------------------------------------------------- */
/* Serving: continuous batching of W1 requests of mixed sizes                */
/* ------------------------------------------------------------------------- */
/*
 * A server owns a worker thread and device-resident plans ("slots") for the
 * size classes it has seen (grid, h, levels, norm, tol).  Requests are queued
 * by w1_submit and started as soon as a slot of their class is free or can be
 * created within the HBM budget (idle slots of other classes are evicted,
 * least recently used first); up to max_slots solves run at once on their own
 * streams, so their work overlaps on the device.  With latency_below = 0 a
 * request's result does not depend on what else is in flight; with
 * latency_below > 0 the kernel choice depends on the load, and results agree
 * to FP32 rounding (W1 within 1e-4, tested).  All calls are thread-safe.  Streams share
 * the context's hardware work queues (8 unless CUDA_DEVICE_MAX_CONNECTIONS is
 * set, up to 32, before CUDA initialises); with more slots than queues, long
 * level solves on one queue delay the launches of the streams that share it.
 */
typedef struct w1_server w1_server;

typedef struct {
    size_t hbm_budget_bytes; /* device memory for slots (plans + input staging); default 40 GiB */
    int max_slots;           /* solves in flight at once; default 32 */
    int max_batch;           /* requests of one class solved together in a slot; default 1 */
    w1_options opt;          /* plan options of every slot */
    int latency_below;       /* while fewer solves than this are in flight, a request goes to a
                                slot whose plan lets the autotuner pick the fastest kernels for
                                one solve alone (w1_options.tune = 1: more SMs per level); at
                                higher load, to a slot with `opt` (throughput); 0 (default): off.
                                Applies when opt.path = 0 and opt.algorithm = 3.  A class may
                                then hold slots of both kinds.  The first latency-tuned slot
                                of a class runs the autotuner on the worker thread (tens of
                                milliseconds per level, once per class and process; the
                                choices are cached): warm each class up with one request. */
} w1_server_config;

typedef struct {
    long long submitted, completed, rejected, queued, in_flight, slots, evictions;
    size_t bytes_in_use;
} w1_server_info;

void w1_server_default_config(w1_server_config* cfg);
/* hbm_budget_bytes = 0 and max_slots <= 0 take the defaults. Uses the current device. */
w1_status w1_server_create(size_t hbm_budget_bytes, int max_slots, w1_server** out);
w1_status w1_server_create_ex(const w1_server_config* cfg, w1_server** out);
/*
 * Queues one request (arguments as w1_plan_create + w1_solve).  rho0, rho1 are
 * device [ny][nx] float32 and must stay valid until the request is finished.
 * Returns W1_ERR_BUDGET if one slot of this class alone exceeds the budget,
 * W1_ERR_SHAPE / W1_ERR_INVALID_ARG for bad arguments.
 */
w1_status w1_submit(w1_server* srv, int nx, int ny, double h, int levels, int norm, double tol, const float* rho0,
                    const float* rho1, uint64_t* ticket);
/* W1_PENDING while queued or running; then the request's own status (as
 * w1_solve) with dist and stats written, and the ticket is released. */
w1_status w1_poll(w1_server* srv, uint64_t ticket, double* dist, w1_stats* stats);
/* w1_poll that also returns the submit-to-finish time measured by the server. */
w1_status w1_poll_latency(w1_server* srv, uint64_t ticket, double* dist, w1_stats* stats, double* latency_s);
/* Blocks until the request finishes or timeout_s passes (<= 0: no limit). */
w1_status w1_wait(w1_server* srv, uint64_t ticket, double timeout_s, double* dist, w1_stats* stats);
w1_status w1_server_query(w1_server* srv, w1_server_info* info);
/* Finishes the solves in flight, fails queued requests, frees every slot. */
w1_status w1_server_destroy(w1_server* srv);
const char* w1_server_last_error(void);

/* ------------------------------------------------------------------------- */
/* Building blocks (device pointers, float32 planes [ny][nx]); used by the   */
/* parity tests and by callers that drive the levels themselves.             */
/* ------------------------------------------------------------------------- */

/*
 * `iters` steps of eq. primaldual in place on (m1, m2, phi) with density rho,
 * step sizes mu, tau, spacing h.  path: 1 shared-memory resident (bands of
 * whole rows in a cluster of up to 16 CTAs: at most 4096 nodes per CTA, or
 * 16384 when nx % 4 == 0 and the band is a multiple of 128 nodes; else
 * W1_ERR_UNSUPPORTED), 2 streaming, 3 temporally blocked streaming
 * (nx and iters multiples of 4).  The four planes must be 16-byte aligned
 * (W1_ERR_INVALID_ARG otherwise).  If fpr_last is not NULL it receives R^k of
 * the last step (FP64 sums).  The boundary flux entries m1[.][nx-1] and
 * m2[ny-1][.] are zero by definition (zero flux); values stored there are
 * ignored and come back as 0.
 */
w1_status w1_cp_steps(int nx, int ny, double h, int norm, float mu, float tau, const float* rho, float* m1,
                      float* m2, float* phi, long long iters, int path, void* stream, double* fpr_last);
/* w1_cp_steps with the cluster size of the resident path chosen by the caller
 * (cluster = 1, 2, 4, 8 or 16 CTAs; 0 picks it as w1_cp_steps does;
 * W1_ERR_UNSUPPORTED if the level does not fit that cluster).  For path 3 the
 * same argument picks the tile variant as w1_options.tile does (0: the first;
 * k in 1..W1_TILE_VARIANTS: variant k - 1; iters must be a multiple of its
 * depth); path 2 ignores it. */
w1_status w1_cp_steps_ex(int nx, int ny, double h, int norm, float mu, float tau, const float* rho, float* m1,
                         float* m2, float* phi, long long iters, int path, int cluster, void* stream,
                         double* fpr_last);

/*
 * Prox-PDHG building blocks (Algorithm 2, eq. pdhg), grids whose sides are
 * powers of two in [2, 1024].  w1_poisson: psi (device [ny][nx]) with
 * -div^h grad psi = r - mean(r) and mean(psi) = 0 (the Neumann Laplacian A_h A_h^*,
 * solved with DCT-II transforms), r and psi may alias.  w1_pdhg_steps: `iters`
 * steps of eq. pdhg in place on (m, phi, phibar) with density rho (zero mean),
 * step sizes mu, tau (the paper takes 1/2); g_last (host, or NULL) receives
 * G^k of eq. pdhg_stop of the last step.  All planes device float32 [ny][nx].
 */
w1_status w1_poisson(int nx, int ny, double h, const float* r, float* psi, void* stream);
w1_status w1_pdhg_steps(int nx, int ny, double h, int norm, float mu, float tau, const float* rho, float* m1,
                        float* m2, float* phi1, float* phi2, float* phibar1, float* phibar2, long long iters,
                        void* stream, double* g_last);

/* coarse[ny/2][nx/2] = mean of each 2x2 block of fine[ny][nx] (density restriction). */
w1_status w1_restrict(int nx, int ny, const float* fine, float* coarse, void* stream);

/* Interpolate (Sec. 3.3, pixel-grid restatement) from a coarse ncx x ncy state
 * to the fine 2ncx x 2ncy state; see the oracle for the rules. */
w1_status w1_prolong(int ncx, int ncy, const float* m1c, const float* m2c, const float* phic, float* m1f,
                     float* m2f, float* phif, void* stream);

/* Statistics of a state (fields w1 (= saddle), primal, saddle, dual, lb, ub,
 * route, res_l1, rho_l1, gmax of *out), rho already balanced; blocks until done. */
w1_status w1_state_stats(int nx, int ny, double h, int norm, const float* rho, const float* m1, const float* m2,
                         const float* phi, void* stream, w1_stats* out);

/*
 * w1_state_stats without allocating device memory.  The paper has no
 * counterpart; this exists for callers that cannot call cudaMalloc: loops
 * that must not pay the implicit device-wide synchronisation of
 * cudaMalloc/cudaFree, frameworks that own all device memory through their own
 * pools (an allocation behind their back breaks their accounting and limits),
 * and services that must run in a fixed, preallocated memory footprint.  Same
 * arguments, results and numbers as w1_state_stats.
 *   - Scratch lives in one file-scope static device array of about 4.2 MB
 *     (control block, partial sums, 2 * W1_NOALLOC_MAX_NODES FP64 masses) that
 *     every GPU loading the library holds until the process exits.
 *   - Grids with more than W1_NOALLOC_MAX_NODES nodes are rejected with
 *     W1_ERR_INVALID_ARG (message in w1_noalloc_last_error()).
 *   - The first call on a device looks up the array's device address with that
 *     device current; make that first call before any stream capture.
 *   - Every call on a device shares the one array, which keeps the last call's
 *     contents (the call clears what must start at zero).  Calls whose work
 *     overlaps on the GPU (other streams, other host threads) race on it:
 *     serialise them.
 *   - Before it returns, the call copies the statistics to the host and
 *     synchronises the stream.
 */
#define W1_NOALLOC_MAX_NODES 262144
w1_status w1_state_stats_noalloc(int nx, int ny, double h, int norm, const float* rho, const float* m1,
                                 const float* m2, const float* phi, void* stream, w1_stats* out);
const char* w1_noalloc_last_error(void);

/* ---------------------------------------------------------------------------
 * Three-dimensional grids.  The discretisation of Sec. 2-3 and Algorithm 3
 * with d = 3: voxel-centre grid nx x ny x nz with spacing h, device arrays
 * [nz][ny][nx] FP32 (x fastest), flux components m1, m2, m3 along x, y, z
 * (the last x-, y-, z-face of the grid carries zero flux), sums weighted by
 * h^3, backward-difference divergence and forward-difference gradient,
 * ||A_h|| <= 2 sqrt(3) / h so mu = tau = theta h / (2 sqrt 3).  A level too
 * large for the on-chip kernels streams each step of eq. primaldual through HBM
 * in one launch (m' recomputed on each voxel's lower neighbours, the new state
 * written beside the old) or two (m' with the mbar extrapolation, then phi');
 * the host reads R^k of eq. pd_stop after every K-th step.  Every pointer is a
 * device pointer owned by the caller (16-byte alignment not required); the
 * calls allocate their own scratch and synchronise the stream before they
 * return.  Errors: W1_ERR_INVALID_ARG (NULL pointer, bad size, unknown norm,
 * bad options), W1_ERR_SHAPE (sizes not divisible by 2^(levels-1)), W1_ERR_MASS,
 * W1_ERR_NOMEM, W1_ERR_CUDA; message in w1_3d_last_error().
 * ------------------------------------------------------------------------- */

/* Algorithm 3 on a 3-D grid.  rho0, rho1: n = nx ny nz densities.  h <= 0 gives
 * 1 / max(nx, ny, nz); levels <= 0 gives Sec. 5's L = log2(1/h) - 3 (at least 1,
 * lowered until every side divides by 2^(L-1) and the coarsest side is >= 2);
 * tol <= 0 gives eq. stop_tol's formula 1e-6/128 (512 h)^2 (the paper states it
 * for 2-D grids; taken unchanged for 3-D); options as for the 2-D solver
 * (check_every 0 = 32; path 0 runs a level on chip (all its steps and stop
 * tests in one launch of one CTA or a cluster of up to 16, each holding at most
 * 4096 voxels in registers or, as wide slabs with each thread's own state in
 * tensor memory, 16384 voxels (a multiple of 128; in a cluster nx ny <= 4096);
 * nx % 4 == 0) where it fits and otherwise with one launch per
 * step and the host testing R^k every K steps; path 1 requires the on-chip
 * kernel (W1_ERR_UNSUPPORTED where a level does not fit); path 2 uses the
 * two-launch step and path 3 the one-launch step on every level (stats->path:
 * 1 on chip, 2 two launches, 3 one launch per step); time_budget_s applies per
 * level; tune,
 * eager and algorithm do not apply).  Writes *dist = f(m) of the
 * finest flux; flux (3n floats: m1, m2, m3 planes) and potential (n floats), when
 * not NULL, receive the finest state; stats: per-level iterations, R^k and eps_l
 * (nx[], ny[] hold the level sizes; the level's nz is nz >> (levels-1-l)),
 * f, the dual value, the certified bracket [lb, ub] with the octree route bound,
 * the masses (sums weighted by h^3).  Returns W1_OK, W1_ERR_NOT_CONVERGED or
 * W1_ERR_TIMEOUT (dist and stats still written), or an error. */
w1_status w1_solve3d(int nx, int ny, int nz, double h, int levels, int norm, double tol,
                     const w1_options* opt, const float* rho0, const float* rho1, void* stream,
                     double* dist, float* flux, float* potential, w1_stats* stats);
/* w1_solve3d keeps its device workspace (level arena, scratch) in a
 * process-wide pool between calls, one per concurrent caller; this frees it
 * (no call may be in flight). */
void w1_3d_release_workspace(void);

/* `iters` steps of eq. primaldual on one 3-D level, in place on m1, m2, m3, phi
 * (zero-mean rho); mu, tau as given.  *fpr_last (may be NULL) = R^k of the last
 * step (0 when iters == 0).  Runs the two-launch step (path 2). */
w1_status w1_cp_steps3d(int nx, int ny, int nz, double h, int norm, float mu, float tau, const float* rho,
                        float* m1, float* m2, float* m3, float* phi, long long iters, void* stream,
                        double* fpr_last);
/* The same with a choice of kernel: path 2 = two launches per step; path 3 = one
 * launch per step (the state alternates with scratch planes and ends in m1, m2,
 * m3, phi; the new state is bitwise path 2's, R^k may differ in rounding); path 1 =
 * every step in one launch on chip (nx % 4 == 0, a cluster of `cluster` CTAs
 * (0: the library's choice) each holding nz / cluster planes: at most 4096
 * voxels, or 16384 as a wide slab (see w1_solve3d); W1_ERR_UNSUPPORTED when
 * the level does not fit); path 1 needs 16-byte aligned planes. */
w1_status w1_cp_steps3d_ex(int nx, int ny, int nz, double h, int norm, float mu, float tau, const float* rho,
                           float* m1, float* m2, float* m3, float* phi, long long iters, int path, int cluster,
                           void* stream, double* fpr_last);

/* Restriction of Algorithm 3 in 3-D: coarse node = mean of its 2x2x2 block;
 * fine is nx x ny x nz (all even), coarse (nx/2)(ny/2)(nz/2).  Asynchronous. */
w1_status w1_restrict3d(int nx, int ny, int nz, const float* fine, float* coarse, void* stream);

/* Interpolate of Sec. 3.3 in 3-D (coarse ncx x ncy x ncz to fine 2ncx x 2ncy x
 * 2ncz): phi trilinear on voxel centres (3/4 own cell, 1/4 the neighbour on the
 * fine voxel's side per axis, clamped at the walls); each flux component copies
 * the coarse face on odd fine faces along its axis, averages the two coarse
 * faces of the cell on even ones, copies across the other axes; zero on the
 * last face.  Asynchronous. */
w1_status w1_prolong3d(int ncx, int ncy, int ncz, const float* m1c, const float* m2c, const float* m3c,
                       const float* phic, float* m1f, float* m2f, float* m3f, float* phif, void* stream);
const char* w1_3d_last_error(void);

/* Text for a status, and the last error message of the calling thread. */
const char* w1_status_string(w1_status s);
const char* w1_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* W1_H_ */
