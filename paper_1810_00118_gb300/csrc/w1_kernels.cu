// w1_kernels.cu -- sm_103a kernels of the multilevel primal-dual W1 solver.
//
// The method (Liu, Yin, Li, Chow, arXiv 1810.00118):
//   Algorithm 1, one step (eq. primaldual, all h^2 weights cancelled):
//     m'   = prox_{mu||.||_p}(m + mu * grad phi)          grad: forward differences
//     mbar = 2 m' - m
//     phi' = phi + tau * (div mbar - rho)                  div: backward differences
//   with the zero-flux boundary of Sec. 2.2 (m1[:, nx-1] = m2[ny-1, :] = 0), and
//   the stop test R^k < eps_l of eq. pd_stop, taken after every K-th step.
//   Algorithm 3 runs it coarse to fine with 2x2 restriction of rho and the
//   Interpolate of Sec. 3.3 (restated for pixel grids).
//
// The step is a memory-bound 5-point stencil (about 30 flops per 28 bytes), so
// no tensor cores are involved.  Two level paths:
//   * resident: a whole level lives on chip in one CTA or one thread-block
//     cluster (bands of rows; halo rows read through distributed shared
//     memory); all steps and stop tests of the level run inside one launch.
//   * streaming: one launch per step over global memory (ping-pong buffers);
//     each warp covers 32 columns and marches up a strip of rows, carrying the
//     row below in registers, prefetching the row above, and exchanging the
//     left/right neighbours by warp shuffles, so every value is read once per
//     step (28 B/node/step).
// Every kernel is batched over the pairs of a plan (same grid for all pairs).
// Reductions are FP64 with a fixed summation order (deterministic).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "w1_device.cuh"
#include "w1_internal.h"

namespace cg = cooperative_groups;

namespace w1 {

// ---------------------------------------------------------------------------
// Prep: rho = rho0 - rho1 (Sec. 2.2), mass check, exact zero mean
// ---------------------------------------------------------------------------

static constexpr int PREP_THREADS = 256;

// Blocks per pair from the grid alone, whatever the batch size, so that every
// pair's sums run in the same order alone and inside a batch (bitwise equal
// results): one per 2048 nodes, at most PREP_BLOCKS_PER_PAIR.  Each block ends
// with a block-wide FP64 sum, so small grids take few blocks.
static constexpr int PREP_BLOCKS_PER_PAIR = 64;
static int prep_blocks_per_pair(int) { return PREP_BLOCKS_PER_PAIR; }
static int prep_blocks(long long n)
{
    const long long b = (n + 2047) / 2048;
    return (int)(b < 1 ? 1 : b > PREP_BLOCKS_PER_PAIR ? PREP_BLOCKS_PER_PAIR : b);
}

// per block: compensated sums (s, c) of r0, r1 and r0 - r1, then the non-finite count
static constexpr int PREP_PART_PER_BLOCK = 7;
size_t prep_part_doubles(int pairs) { return (size_t)prep_blocks_per_pair(pairs) * pairs * PREP_PART_PER_BLOCK; }

__global__ void __launch_bounds__(PREP_THREADS) k_prep_reduce(const float* __restrict__ r0,
                                                              const float* __restrict__ r1, long long n, int nbatch,
                                                              double h, Ctl* ctls, double* part)
{
    __shared__ double sh[2 * 3 * PREP_THREADS];
    __shared__ bool last;
    const int pair = blockIdx.y;
    Ctl* ctl = ctls + pair;
    if (pair >= nbatch) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            ctl->error = 2;
            ctl->timeout = 0;
            ctl->counter = 0;
        }
        return;
    }
    r0 += (size_t)pair * n;
    r1 += (size_t)pair * n;
    double* pp = part + (size_t)pair * gridDim.x * PREP_PART_PER_BLOCK;
    // compensated sums of r0, r1 and r0 - r1 (each difference of two FP32 values is exact in FP64)
    CSum v[3];
    unsigned bad = 0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        float a = r0[k], b = r1[k];
        if (!isfinite(a) || !isfinite(b)) ++bad;
        v[0].add(a);
        v[1].add(b);
        v[2].add(__dsub_rn((double)a, (double)b));
    }
    block_csum_sh<3>(v, sh);
    double nb[1] = {(double)bad};
    block_sum<1>(nb, sh);
    if (threadIdx.x == 0) {
        for (int c = 0; c < 3; ++c) {
            pp[blockIdx.x * PREP_PART_PER_BLOCK + 2 * c] = v[c].s;
            pp[blockIdx.x * PREP_PART_PER_BLOCK + 2 * c + 1] = v[c].c;
        }
        pp[blockIdx.x * PREP_PART_PER_BLOCK + 6] = nb[0];
        __threadfence();
        last = (atomicAdd(&ctl->counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    CSum t[3];
    double nf[1] = {0.0};
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
        const volatile double* q = pp + (size_t)b * PREP_PART_PER_BLOCK;
        for (int c = 0; c < 3; ++c) {
            CSum x;
            x.s = q[2 * c];
            x.c = q[2 * c + 1];
            t[c].add(x);
        }
        nf[0] += q[6];
    }
    block_csum_sh<3>(t, sh);
    block_sum<1>(nf, sh);
    if (threadIdx.x == 0) {
        const double M0 = t[0].value() * h * h, M1 = t[1].value() * h * h;
        ctl->mass0 = M0;
        ctl->mass1 = M1;
        ctl->mean = t[2].value() / (double)n;
        int bad_in = (nf[0] > 0.0) || !(fabs(M0 - M1) <= 1e-6 * fmax(fabs(M0), fabs(M1)));
        ctl->error = bad_in;
        ctl->timeout = 0;
        ctl->counter = 0;
    }
}

__global__ void k_prep_apply(const float* __restrict__ r0, const float* __restrict__ r1, long long n, int nbatch,
                             const Ctl* __restrict__ ctls, float* __restrict__ rho)
{
    const int pair = blockIdx.y;
    if (pair >= nbatch) return;
    const double mean = ctls[pair].mean;
    const size_t off = (size_t)pair * n;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        rho[off + k] = (float)(((double)r0[off + k] - (double)r1[off + k]) - mean);
}

cudaError_t launch_prep(const float* r0, const float* r1, long long n, int nbatch, int pairs, double h, Ctl* ctl,
                        double* part, float* rho, cudaStream_t s)
{
    const int bpp = prep_blocks(n);
    k_prep_reduce<<<dim3(bpp, pairs), PREP_THREADS, 0, s>>>(r0, r1, n, nbatch, h, ctl, part);
    k_prep_apply<<<dim3(2 * bpp, pairs), 256, 0, s>>>(r0, r1, n, nbatch, ctl, rho);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Restriction (2x2 block mean) and Interpolate (Sec. 3.3, pixel-grid reading)
// ---------------------------------------------------------------------------

// coarse node (I, J) = mean of its 2x2 block of fine nodes (pointers at one pair's planes)
__device__ __forceinline__ void restrict_node(const float* __restrict__ f, int nx, float* __restrict__ c, int ncx, int I,
                                              int J)
{
    const float* r0 = f + (size_t)(2 * J) * nx + 2 * I;
    const float* r1 = r0 + nx;
    c[(size_t)J * ncx + I] = 0.25f * ((r0[0] + r0[1]) + (r1[0] + r1[1]));
}

__global__ void k_restrict(const float* __restrict__ f, int nx, int ny, float* __restrict__ c, const Ctl* ctls)
{
    const int ncx = nx / 2, ncy = ny / 2;
    const int pair = blockIdx.z;
    if (ctls && ctls[pair].error) return;
    const int I = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y * blockDim.y + threadIdx.y;
    if (I >= ncx || J >= ncy) return;
    restrict_node(f + (size_t)pair * nx * ny, nx, c + (size_t)pair * ncx * ncy, ncx, I, J);
}

cudaError_t launch_restrict(const float* fine, int nx, int ny, float* coarse, int pairs, const Ctl* ctl,
                            cudaStream_t s)
{
    dim3 b(32, 8), g((nx / 2 + 31) / 32, (ny / 2 + 7) / 8, pairs);
    k_restrict<<<g, b, 0, s>>>(fine, nx, ny, coarse, ctl);
    return cudaGetLastError();
}

// phi: bilinear on cell centres (3/4 own coarse cell, 1/4 the neighbour on the
// fine node's side, clamped); m1: odd fine x-edges copy the coarse x-edge they
// lie on, even ones average the coarse x-edges around their coarse cell, rows
// copy; m2 likewise with the axes exchanged.
// fine node (i, j) from the coarse state (pointers at one pair's planes)
__device__ __forceinline__ void prolong_node(int ncx, int ncy, const float* __restrict__ m1c,
                                             const float* __restrict__ m2c, const float* __restrict__ phic,
                                             float* __restrict__ m1f, float* __restrict__ m2f,
                                             float* __restrict__ phif, int i, int j)
{
    const int nx = 2 * ncx, ny = 2 * ncy;
    const int I = i >> 1, J = j >> 1;
    const int In = min(max((i & 1) ? I + 1 : I - 1, 0), ncx - 1);
    const int Jn = min(max((j & 1) ? J + 1 : J - 1, 0), ncy - 1);
    const float* rowJ = phic + (size_t)J * ncx;
    const float* rowN = phic + (size_t)Jn * ncx;
    float p = 0.5625f * rowJ[I] + 0.1875f * rowJ[In] + 0.1875f * rowN[I] + 0.0625f * rowN[In];
    float v1, v2;
    if (i & 1) {
        v1 = m1c[(size_t)J * ncx + I];
    } else {
        float left = I > 0 ? m1c[(size_t)J * ncx + I - 1] : 0.f;
        v1 = 0.5f * (left + m1c[(size_t)J * ncx + I]);
    }
    if (i == nx - 1) v1 = 0.f;
    if (j & 1) {
        v2 = m2c[(size_t)J * ncx + I];
    } else {
        float below = J > 0 ? m2c[(size_t)(J - 1) * ncx + I] : 0.f;
        v2 = 0.5f * (below + m2c[(size_t)J * ncx + I]);
    }
    if (j == ny - 1) v2 = 0.f;
    const size_t k = (size_t)j * nx + i;
    phif[k] = p;
    m1f[k] = v1;
    m2f[k] = v2;
}

__global__ void k_prolong(int ncx, int ncy, const float* __restrict__ m1c, const float* __restrict__ m2c,
                          const float* __restrict__ phic, float* __restrict__ m1f, float* __restrict__ m2f,
                          float* __restrict__ phif, const Ctl* ctls)
{
    const int nx = 2 * ncx, ny = 2 * ncy;
    const int pair = blockIdx.z;
    if (ctls && ctls[pair].error) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= nx || j >= ny) return;
    const size_t co = (size_t)pair * ncx * ncy, fo = (size_t)pair * nx * ny;
    prolong_node(ncx, ncy, m1c + co, m2c + co, phic + co, m1f + fo, m2f + fo, phif + fo, i, j);
}

cudaError_t launch_prolong(int ncx, int ncy, const float* m1c, const float* m2c, const float* phic, float* m1f,
                           float* m2f, float* phif, int pairs, const Ctl* ctl, cudaStream_t s)
{
    dim3 b(32, 8), g((2 * ncx + 31) / 32, (2 * ncy + 7) / 8, pairs);
    k_prolong<<<g, b, 0, s>>>(ncx, ncy, m1c, m2c, phic, m1f, m2f, phif, ctl);
    return cudaGetLastError();
}

__global__ void k_level_begin(Ctl* ctls, int level, int pairs)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= pairs) return;
    Ctl* c = ctls + p;
    c->iters[level] = 0;
    c->fpr[level] = 0.0;
    c->conv[level] = 0;
    c->t_start[level] = globaltimer();
    c->active = c->error ? 0 : 1;
}

cudaError_t launch_level_begin(Ctl* ctl, int level, int pairs, cudaStream_t s)
{
    k_level_begin<<<(pairs + 127) / 128, 128, 0, s>>>(ctl, level, pairs);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Streaming step (one step of eq. primaldual over global memory)
// ---------------------------------------------------------------------------

static constexpr int STEP_THREADS = 256;  // 8 warps stacked in y

int stream_rows_auto(int nx, int ny, int)
{
    // enough blocks for ~4 waves of 152 SMs for one pair, marching at most 16
    // rows per thread; independent of the batch size so that each pair's R^k is
    // summed in the same order alone and inside a batch
    long long colblocks = (nx + 31) / 32;
    long long r = (long long)ny * colblocks / (8LL * 152 * 4);
    if (r < 2) r = 2;
    if (r > 16) r = 16;
    return (int)r;
}

dim3 stream_grid(int nx, int ny, int rows, int pairs)
{
    return dim3((nx + 31) / 32, (ny + 8 * rows - 1) / (8 * rows), pairs);
}

size_t step_part_doubles(int nx, int ny, int rows, int pairs)
{
    dim3 g = stream_grid(nx, ny, rows, pairs);
    return (size_t)g.x * g.y * g.z * 3;
}

template <int NORM, bool CHECK>
__global__ void __launch_bounds__(STEP_THREADS) k_step(StepArgs a)
{
    const IterArgs& P = a.it;
    const int pair = blockIdx.z;
    Ctl* pc = P.ctl ? P.ctl + pair : nullptr;
    // a pair that was rejected, is an unused slot, or has converged does no work
    if (pc && (pc->error || (a.use_cond && !pc->active))) return;  // uniform over the pair's blocks
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nx = P.nx, ny = P.ny;
    const int i = blockIdx.x * 32 + lane;
    const int j0 = (blockIdx.y * (STEP_THREADS / 32) + warp) * a.rows;
    const bool act = i < nx;
    const float mu = P.mu, tau = P.tau;
    const float cm = P.mu * P.ih, ct = P.tau * P.ih;  // mu / h, tau / h
    const size_t off = (size_t)pair * P.stride;
    // test-step sums: FP32 terms and per-thread partials (a strip of rows), FP64
    // across threads and blocks (FP64 is a small fraction of FP32 throughput here)
    float sa = 0.f, sb = 0.f, sc = 0.f;
    if (j0 < ny) {
        const int j1 = min(j0 + a.rows, ny);
        const float* __restrict__ phi = a.phi + off;
        const float* __restrict__ m1 = a.m1 + off;
        const float* __restrict__ m2 = a.m2 + off;
        const float* __restrict__ rho = a.rho + off;
        float* __restrict__ m1o = a.m1o + off;
        float* __restrict__ m2o = a.m2o + off;
        float* __restrict__ phio = a.phio + off;
        auto at = [nx](int j, int ii) { return (size_t)j * nx + ii; };
        float pc_ = act ? __ldg(phi + at(j0, i)) : 0.f;
        // mbar2 and dm2 of the node below the strip (row j0 - 1)
        float b2b = 0.f;
        float d2b = 0.f;
        if (j0 > 0) {
            float pb = act ? __ldg(phi + at(j0 - 1, i)) : 0.f;
            float c2 = act ? __ldg(m2 + at(j0 - 1, i)) : 0.f;
            const float v2 = fmaf(cm, pc_ - pb, c2);
            float o1 = 0.f, o2;
            if (NORM == W1_NORM_L1) {
                o2 = soft(v2, mu);
            } else {
                float pbr = __shfl_down_sync(FULL, pb, 1);
                if (lane == 31 && i + 1 < nx) pbr = __ldg(phi + at(j0 - 1, i + 1));
                const float c1 = act ? __ldg(m1 + at(j0 - 1, i)) : 0.f;
                const float v1 = (i < nx - 1) ? fmaf(cm, pbr - pb, c1) : 0.f;
                prox<NORM>(v1, v2, mu, o1, o2);
            }
            (void)o1;
            b2b = 2.f * o2 - c2;
            d2b = o2 - c2;
        }
        // row j's values are loaded one row ahead (software pipelining)
        float nu = (act && j0 + 1 < ny) ? __ldg(phi + at(j0 + 1, i)) : 0.f;
        float na1 = act ? __ldg(m1 + at(j0, i)) : 0.f;
        float na2 = act ? __ldg(m2 + at(j0, i)) : 0.f;
        float nr = act ? __ldg(rho + at(j0, i)) : 0.f;
        for (int j = j0; j < j1; ++j) {
            const float pu = nu, a1 = na1, a2 = na2, r = nr;
            if (j + 1 < j1) {
                nu = (act && j + 2 < ny) ? __ldg(phi + at(j + 2, i)) : 0.f;
                na1 = act ? __ldg(m1 + at(j + 1, i)) : 0.f;
                na2 = act ? __ldg(m2 + at(j + 1, i)) : 0.f;
                nr = act ? __ldg(rho + at(j + 1, i)) : 0.f;
            }
            float pr = __shfl_down_sync(FULL, pc_, 1);
            if (lane == 31 && i + 1 < nx) pr = __ldg(phi + at(j, i + 1));
            // pinned entries (last column, top row) enter as zero and stay zero
            const float v1 = (i < nx - 1) ? fmaf(cm, pr - pc_, a1) : 0.f;
            const float v2 = (j < ny - 1) ? fmaf(cm, pu - pc_, a2) : 0.f;
            float n1, n2;
            prox<NORM>(v1, v2, mu, n1, n2);
            if (i >= nx - 1) n1 = 0.f;
            if (j == ny - 1) n2 = 0.f;
            const float b1 = 2.f * n1 - a1, b2 = 2.f * n2 - a2;
            float b1l = __shfl_up_sync(FULL, b1, 1);
            float d1l = 0.f;
            if (CHECK) d1l = __shfl_up_sync(FULL, n1 - a1, 1);
            if (lane == 0) {
                if (i > 0) {
                    // the left neighbour belongs to the previous warp: recompute its m1'
                    const float ql = __ldg(phi + at(j, i - 1));
                    const float c1 = __ldg(m1 + at(j, i - 1));
                    const float vl1 = fmaf(cm, pc_ - ql, c1);
                    float o1, o2;
                    if (NORM == W1_NORM_L1) {
                        o1 = soft(vl1, mu);
                    } else {
                        const float qlu = (j + 1 < ny) ? __ldg(phi + at(j + 1, i - 1)) : 0.f;
                        const float c2 = __ldg(m2 + at(j, i - 1));
                        const float vl2 = (j < ny - 1) ? fmaf(cm, qlu - ql, c2) : 0.f;
                        prox<NORM>(vl1, vl2, mu, o1, o2);
                    }
                    b1l = 2.f * o1 - c1;
                    d1l = o1 - c1;
                } else {
                    b1l = 0.f;
                    d1l = 0.f;
                }
            }
            const float dv = (b1 - b1l) + (b2 - b2b);  // h div mbar
            const float pn = fmaf(ct, dv, fmaf(-tau, r, pc_));
            if (act) {
                m1o[at(j, i)] = n1;
                m2o[at(j, i)] = n2;
                phio[at(j, i)] = pn;
            }
            if (CHECK && act) {
                const float e1 = n1 - a1, e2 = n2 - a2;
                const float ep = pn - pc_;
                const float dd = (e1 - d1l) + (e2 - d2b);  // h div dm
                sa = fmaf(e1, e1, fmaf(e2, e2, sa));
                sb = fmaf(ep, ep, sb);
                sc = fmaf(ep, dd, sc);
                d2b = e2;
            }
            b2b = b2;
            pc_ = pu;
        }
    }
    if (!CHECK) return;

    // R^k = (|dm|^2 / mu + |dphi|^2 / tau - 2 <dphi, div dm>) h^2   (eq. pd_stop)
    __shared__ double sh[64 * 3];
    __shared__ bool last;
    double v[3];
    ff_block_sum3(sa, sb, sc, reinterpret_cast<float*>(sh), v);
    const int nblk = gridDim.x * gridDim.y;
    const int bid = blockIdx.y * gridDim.x + blockIdx.x;
    double* pp = a.part + (size_t)pair * nblk * 3;
    if (threadIdx.x == 0) {
        pp[bid * 3 + 0] = v[0];
        pp[bid * 3 + 1] = v[1];
        pp[bid * 3 + 2] = v[2];
        __threadfence();
        last = (atomicAdd(&pc->counter, 1u) == (unsigned)nblk - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    CSum t[3];
    for (int b = threadIdx.x; b < nblk; b += blockDim.x)
        for (int c = 0; c < 3; ++c) t[c].add(((volatile double*)pp)[b * 3 + c]);
    block_csum<3>(t, sh);
    if (threadIdx.x == 0) {
        const double h2 = P.h * P.h;
        const double R = (t[0].value() / (double)P.mu + t[1].value() / (double)P.tau - 2.0 * (t[2].value() / P.h)) * h2;
        pc->counter = 0;
        if (P.fpr_out) P.fpr_out[pair] = R;
        if (a.use_cond) {
            const long long it = pc->iters[P.level] + P.K;
            pc->iters[P.level] = it;
            pc->fpr[P.level] = R;
            const int conv = R < P.tol;
            pc->conv[P.level] = conv;
            const bool late = (globaltimer() - pc->t_start[P.level]) > P.budget_ns;
            if (late && !conv) pc->timeout = 1;
            if (conv || it >= P.cap || late) pc->active = 0;
        }
    }
}

cudaError_t launch_step(int norm, bool check, const StepArgs& a, cudaStream_t s)
{
    dim3 g = stream_grid(a.it.nx, a.it.ny, a.rows, a.pairs);
    if (norm == W1_NORM_L1) {
        if (check) k_step<W1_NORM_L1, true><<<g, STEP_THREADS, 0, s>>>(a);
        else k_step<W1_NORM_L1, false><<<g, STEP_THREADS, 0, s>>>(a);
    } else if (norm == W1_NORM_L2) {
        if (check) k_step<W1_NORM_L2, true><<<g, STEP_THREADS, 0, s>>>(a);
        else k_step<W1_NORM_L2, false><<<g, STEP_THREADS, 0, s>>>(a);
    } else {
        if (check) k_step<W1_NORM_LINF, true><<<g, STEP_THREADS, 0, s>>>(a);
        else k_step<W1_NORM_LINF, false><<<g, STEP_THREADS, 0, s>>>(a);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Temporally blocked streaming step: TB steps per launch
// ---------------------------------------------------------------------------
//
// Each CTA loads a tile of (TBX + 2 TB) x (TBY + 2 TB) nodes (its TBX x TBY
// interior plus a halo of TB on every side) into shared memory, runs TB steps
// of eq. primaldual there with four consecutive nodes of a row per thread, and
// writes the interior back.  A wrong value at the tile's edge moves inwards by
// at most one node per step, so after TB steps the interior is exact.  Nodes
// outside the grid are loaded as zeros and never influence a node of the grid
// (the zero-flux boundary conditions test global indices).  On a test launch
// the last step forms the interior nodes' share of R^k, summed per pair as in
// k_step.  Global traffic per step: (16 B x tile/interior + 12 B) / TB per node.

// The tile (TBX x TBY interior nodes) and the depth TB (steps per launch) are
// compile-time parameters of each instantiation; the plan (or the autotuner)
// picks one of TB_SHAPES per level.  Wider tiles waste less on halos, deeper
// ones read global memory less often, at the cost of more halo work per step.
struct TbShape {
    int x, y, t;
};
static constexpr TbShape TB_SHAPES[W1_TILE_VARIANTS] = {{64, 32, 4}, {128, 16, 4}, {32, 64, 4}, {64, 32, 8}, {32, 32, 8}};
template <int TBX, int TBY, int TB>
struct TbGeom {
    static_assert(TB % 4 == 0 && TBX % 4 == 0, "runs of four nodes must not straddle the tile's interior edge");
    static constexpr int TLW = TBX + 2 * TB, TLH = TBY + 2 * TB, TLN = TLW * TLH;
    static constexpr int THREADS = ((TLN / 4 + 31) / 32) * 32;
    static_assert(THREADS <= 1024, "one thread per run of four tile nodes");
    static constexpr size_t SMEM_PLAIN = 3 * TLN * sizeof(float), SMEM_CHECK = 5 * TLN * sizeof(float);
};

static int tile_index(int tile) { return (tile >= 0 && tile < W1_TILE_VARIANTS) ? tile : 0; }
dim3 tblock_grid(int nx, int ny, int pairs, int tile)
{
    const TbShape& sh = TB_SHAPES[tile_index(tile)];
    return dim3((nx + sh.x - 1) / sh.x, (ny + sh.y - 1) / sh.y, pairs);
}
size_t tblock_part_doubles(int nx, int ny, int pairs)
{
    size_t m = 0;
    for (int k = 0; k < W1_TILE_VARIANTS; ++k) {
        dim3 g = tblock_grid(nx, ny, pairs, k);
        const size_t v = (size_t)g.x * g.y * g.z * 3;
        if (v > m) m = v;
    }
    return m;
}
int tblock_depth(int tile) { return TB_SHAPES[tile_index(tile)].t; }

template <int NORM, bool CHECK, int TBX, int TBY, int TB>
__global__ void __launch_bounds__(TbGeom<TBX, TBY, TB>::THREADS) k_tblock(StepArgs a)
{
    constexpr int TLW = TbGeom<TBX, TBY, TB>::TLW, TLH = TbGeom<TBX, TBY, TB>::TLH, TLN = TbGeom<TBX, TBY, TB>::TLN;
    const IterArgs& P = a.it;
    const int pair = blockIdx.z;
    Ctl* pc = P.ctl ? P.ctl + pair : nullptr;
    if (pc && (pc->error || (a.use_cond && !pc->active))) return;  // uniform over the pair's blocks
    const int nx = P.nx, ny = P.ny;
    const int X0 = blockIdx.x * TBX - TB, Y0 = blockIdx.y * TBY - TB;  // tile origin (may be negative)
    extern __shared__ __align__(16) unsigned char tb_smem[];
    float* ph = reinterpret_cast<float*>(tb_smem);
    float* s1 = ph + TLN;
    float* s2 = s1 + TLN;
    float* e1s = s2 + TLN;  // test launches only
    float* e2s = e1s + TLN;
    const size_t off = (size_t)pair * P.stride;
    const float mu = P.mu, tau = P.tau;
    const float cm = P.mu * P.ih, ct = P.tau * P.ih;  // mu / h, tau / h
    const int t = threadIdx.x;
    const bool own = t < TLN / 4;
    const int W = TLW / 4;
    const int jl = own ? t / W : 0;
    const int il = own ? 4 * (t - jl * W) : 0;
    const int idx = jl * TLW + il;
    const int gj = Y0 + jl, gi0 = X0 + il;
    const bool row_in = gj >= 0 && gj < ny;
    // nx % 4 == 0 and gi0 % 4 == 0: a run of four lies wholly inside or outside the grid
    const bool run_in = own && row_in && gi0 >= 0 && gi0 < nx;
    float m1[4], m2[4], pv[4], rv[4], Dv[4];
    {
        float4 x1 = make_float4(0.f, 0.f, 0.f, 0.f), x2 = x1, xp = x1, xr = x1;
        if (run_in) {
            const size_t g = off + (size_t)gj * nx + gi0;
            x1 = __ldg(reinterpret_cast<const float4*>(a.m1 + g));
            x2 = __ldg(reinterpret_cast<const float4*>(a.m2 + g));
            xp = __ldg(reinterpret_cast<const float4*>(a.phi + g));
            xr = __ldg(reinterpret_cast<const float4*>(a.rho + g));
        }
        m1[0] = x1.x; m1[1] = x1.y; m1[2] = x1.z; m1[3] = x1.w;
        m2[0] = x2.x; m2[1] = x2.y; m2[2] = x2.z; m2[3] = x2.w;
        pv[0] = xp.x; pv[1] = xp.y; pv[2] = xp.z; pv[3] = xp.w;
        rv[0] = xr.x; rv[1] = xr.y; rv[2] = xr.z; rv[3] = xr.w;
    }
    if (own) {
        *reinterpret_cast<float4*>(ph + idx) = make_float4(pv[0], pv[1], pv[2], pv[3]);
        *reinterpret_cast<float4*>(s1 + idx) = make_float4(m1[0], m1[1], m1[2], m1[3]);
        *reinterpret_cast<float4*>(s2 + idx) = make_float4(m2[0], m2[1], m2[2], m2[3]);
    }
    __syncthreads();
    if (own) {  // D^0 = h div m^0 (wrong on the tile's first column and row, as it should be)
        const float l = il > 0 ? s1[idx - 1] : 0.f;
        const float4 b = jl > 0 ? *reinterpret_cast<const float4*>(s2 + idx - TLW) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float bb[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int gi = gi0 + c;
            const float left = c ? m1[c - 1] : l;
            Dv[c] = ((gi < nx - 1 ? m1[c] : 0.f) - (gi > 0 ? left : 0.f)) + ((gj < ny - 1 ? m2[c] : 0.f) - (gj > 0 ? bb[c] : 0.f));
        }
    }
    __syncthreads();
    float sa = 0.f, sb = 0.f, sc = 0.f;  // FP32 terms and per-thread partials, FP64 across threads
    const bool interior_row = jl >= TB && jl < TB + TBY && row_in;
#pragma unroll 1
    for (int step = 0; step < TB; ++step) {
        const bool last = CHECK && step == TB - 1;
        if (own) {
            float up[4] = {0.f, 0.f, 0.f, 0.f};
            if (jl < TLH - 1) {
                const float4 u = *reinterpret_cast<const float4*>(ph + idx + TLW);
                up[0] = u.x; up[1] = u.y; up[2] = u.z; up[3] = u.w;
            }
            const float right = il + 4 < TLW ? ph[idx + 4] : 0.f;
            float n1[4], n2[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                // pinned entries (last column, top row) and nodes past them: v = 0 gives m' = 0
                const int gi = gi0 + c;
                const float pr_ = c < 3 ? pv[c + 1] : right;
                const float v1 = gi < nx - 1 ? fmaf(cm, pr_ - pv[c], m1[c]) : 0.f;
                const float v2 = gj < ny - 1 ? fmaf(cm, up[c] - pv[c], m2[c]) : 0.f;
                prox<NORM>(v1, v2, mu, n1[c], n2[c]);
            }
            if (last) {
                float d1[4], d2[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    d1[c] = n1[c] - m1[c];
                    d2[c] = n2[c] - m2[c];
                    const int ci = il + c;
                    if (interior_row && ci >= TB && ci < TB + TBX && gi0 + c < nx)
                        sa = fmaf(d1[c], d1[c], fmaf(d2[c], d2[c], sa));
                }
                *reinterpret_cast<float4*>(e1s + idx) = make_float4(d1[0], d1[1], d1[2], d1[3]);
                *reinterpret_cast<float4*>(e2s + idx) = make_float4(d2[0], d2[1], d2[2], d2[3]);
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                m1[c] = n1[c];
                m2[c] = n2[c];
            }
            *reinterpret_cast<float4*>(s1 + idx) = make_float4(n1[0], n1[1], n1[2], n1[3]);
            *reinterpret_cast<float4*>(s2 + idx) = make_float4(n2[0], n2[1], n2[2], n2[3]);
        }
        __syncthreads();
        if (own) {
            const float l = il > 0 ? s1[idx - 1] : 0.f;
            const float4 b = jl > 0 ? *reinterpret_cast<const float4*>(s2 + idx - TLW) : make_float4(0.f, 0.f, 0.f, 0.f);
            const float bb[4] = {b.x, b.y, b.z, b.w};
            float pn[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int gi = gi0 + c;
                const float left = c ? m1[c - 1] : l;
                const float Dn = (m1[c] - (gi > 0 ? left : 0.f)) + (m2[c] - (gj > 0 ? bb[c] : 0.f));
                pn[c] = fmaf(ct, fmaf(2.f, Dn, -Dv[c]), fmaf(-tau, rv[c], pv[c]));
                Dv[c] = Dn;
            }
            if (last) {
                const float4 e1 = *reinterpret_cast<const float4*>(e1s + idx);
                const float4 e2 = *reinterpret_cast<const float4*>(e2s + idx);
                const float el = il > 0 ? e1s[idx - 1] : 0.f;
                const float4 eb = jl > 0 ? *reinterpret_cast<const float4*>(e2s + idx - TLW) : make_float4(0.f, 0.f, 0.f, 0.f);
                const float a1[4] = {e1.x, e1.y, e1.z, e1.w}, a2[4] = {e2.x, e2.y, e2.z, e2.w};
                const float bl[4] = {eb.x, eb.y, eb.z, eb.w};
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int ci = il + c, gi = gi0 + c;
                    if (!(interior_row && ci >= TB && ci < TB + TBX && gi < nx)) continue;
                    const float left = c ? a1[c - 1] : (gi > 0 ? el : 0.f);
                    const float below = gj > 0 ? bl[c] : 0.f;
                    const float dd = (a1[c] - left) + (a2[c] - below);  // h div dm
                    const float ep = pn[c] - pv[c];
                    sb = fmaf(ep, ep, sb);
                    sc = fmaf(ep, dd, sc);
                }
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) pv[c] = pn[c];
            *reinterpret_cast<float4*>(ph + idx) = make_float4(pn[0], pn[1], pn[2], pn[3]);
        }
        __syncthreads();
    }
    // write the interior (TB % 4 == 0: a run is wholly interior or wholly halo)
    if (run_in && interior_row && il >= TB && il < TB + TBX) {
        const size_t g = off + (size_t)gj * nx + gi0;
        *reinterpret_cast<float4*>(a.m1o + g) = make_float4(m1[0], m1[1], m1[2], m1[3]);
        *reinterpret_cast<float4*>(a.m2o + g) = make_float4(m2[0], m2[1], m2[2], m2[3]);
        *reinterpret_cast<float4*>(a.phio + g) = make_float4(pv[0], pv[1], pv[2], pv[3]);
    }
    if (!CHECK) return;
    __shared__ double sh[64 * 3];
    __shared__ bool lastblk;
    double v[3];
    ff_block_sum3(sa, sb, sc, reinterpret_cast<float*>(sh), v);
    const int nblk = gridDim.x * gridDim.y;
    const int bid = blockIdx.y * gridDim.x + blockIdx.x;
    double* pp = a.part + (size_t)pair * nblk * 3;
    if (t == 0) {
        pp[bid * 3 + 0] = v[0];
        pp[bid * 3 + 1] = v[1];
        pp[bid * 3 + 2] = v[2];
        __threadfence();
        lastblk = (atomicAdd(&pc->counter, 1u) == (unsigned)nblk - 1);
    }
    __syncthreads();
    if (!lastblk) return;
    __threadfence();
    CSum tt[3];
    for (int b = t; b < nblk; b += blockDim.x)
        for (int c = 0; c < 3; ++c) tt[c].add(((volatile double*)pp)[b * 3 + c]);
    block_csum<3>(tt, sh);
    if (t == 0) {
        const double h2 = P.h * P.h;
        const double R =
            (tt[0].value() / (double)P.mu + tt[1].value() / (double)P.tau - 2.0 * (tt[2].value() / P.h)) * h2;
        pc->counter = 0;
        if (P.fpr_out) P.fpr_out[pair] = R;
        if (a.use_cond) {
            const long long it = pc->iters[P.level] + P.K;
            pc->iters[P.level] = it;
            pc->fpr[P.level] = R;
            const int conv = R < P.tol;
            pc->conv[P.level] = conv;
            const bool late = (globaltimer() - pc->t_start[P.level]) > P.budget_ns;
            if (late && !conv) pc->timeout = 1;
            if (conv || it >= P.cap || late) pc->active = 0;
        }
    }
}

template <int NORM, bool CHECK, int X, int Y, int T>
static cudaError_t tb_attr()
{
    return cudaFuncSetAttribute(k_tblock<NORM, CHECK, X, Y, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(CHECK ? TbGeom<X, Y, T>::SMEM_CHECK : TbGeom<X, Y, T>::SMEM_PLAIN));
}
template <int X, int Y, int T>
static cudaError_t tb_attr_all()
{
    cudaError_t e;
    if ((e = tb_attr<W1_NORM_L1, true, X, Y, T>()) != cudaSuccess) return e;
    if ((e = tb_attr<W1_NORM_L1, false, X, Y, T>()) != cudaSuccess) return e;
    if ((e = tb_attr<W1_NORM_L2, true, X, Y, T>()) != cudaSuccess) return e;
    if ((e = tb_attr<W1_NORM_L2, false, X, Y, T>()) != cudaSuccess) return e;
    if ((e = tb_attr<W1_NORM_LINF, true, X, Y, T>()) != cudaSuccess) return e;
    return tb_attr<W1_NORM_LINF, false, X, Y, T>();
}

cudaError_t tblock_prepare()
{
    cudaError_t e;
    if ((e = tb_attr_all<64, 32, 4>()) != cudaSuccess) return e;
    if ((e = tb_attr_all<128, 16, 4>()) != cudaSuccess) return e;
    if ((e = tb_attr_all<32, 64, 4>()) != cudaSuccess) return e;
    if ((e = tb_attr_all<64, 32, 8>()) != cudaSuccess) return e;
    return tb_attr_all<32, 32, 8>();
}

template <int X, int Y, int T>
static void tb_launch(int norm, bool check, const StepArgs& a, cudaStream_t s)
{
    using G = TbGeom<X, Y, T>;
    const TbShape sh{X, Y, T};
    const dim3 g((a.it.nx + sh.x - 1) / sh.x, (a.it.ny + sh.y - 1) / sh.y, a.pairs);
    if (norm == W1_NORM_L1) {
        if (check) k_tblock<W1_NORM_L1, true, X, Y, T><<<g, G::THREADS, G::SMEM_CHECK, s>>>(a);
        else k_tblock<W1_NORM_L1, false, X, Y, T><<<g, G::THREADS, G::SMEM_PLAIN, s>>>(a);
    } else if (norm == W1_NORM_L2) {
        if (check) k_tblock<W1_NORM_L2, true, X, Y, T><<<g, G::THREADS, G::SMEM_CHECK, s>>>(a);
        else k_tblock<W1_NORM_L2, false, X, Y, T><<<g, G::THREADS, G::SMEM_PLAIN, s>>>(a);
    } else {
        if (check) k_tblock<W1_NORM_LINF, true, X, Y, T><<<g, G::THREADS, G::SMEM_CHECK, s>>>(a);
        else k_tblock<W1_NORM_LINF, false, X, Y, T><<<g, G::THREADS, G::SMEM_PLAIN, s>>>(a);
    }
}

cudaError_t launch_tblock(int norm, bool check, const StepArgs& a, cudaStream_t s)
{
    switch (tile_index(a.tile)) {
    case 1: tb_launch<128, 16, 4>(norm, check, a, s); break;
    case 2: tb_launch<32, 64, 4>(norm, check, a, s); break;
    case 3: tb_launch<64, 32, 8>(norm, check, a, s); break;
    case 4: tb_launch<32, 32, 8>(norm, check, a, s); break;
    default: tb_launch<64, 32, 4>(norm, check, a, s); break;
    }
    static_assert(W1_TILE_VARIANTS == 5, "one case per entry of TB_SHAPES");
    return cudaGetLastError();
}

__global__ void k_decide(const Ctl* __restrict__ ctls, int pairs, cudaGraphConditionalHandle cond)
{
    int any = 0;
    for (int p = threadIdx.x; p < pairs; p += blockDim.x) any |= ctls[p].active;
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) cudaGraphSetConditional(cond, any ? 1u : 0u);
}

cudaError_t launch_decide(const Ctl* ctl, int pairs, cudaGraphConditionalHandle cond, cudaStream_t s)
{
    k_decide<<<1, 256, 0, s>>>(ctl, pairs, cond);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Resident level solver: Algorithm 1 to its stop test inside one launch
// ---------------------------------------------------------------------------
//
// A cluster of C CTAs holds one pair's level; CTA r owns rows
// [r*ny/C, (r+1)*ny/C).  Shared memory holds the band: phi and m (what
// neighbours read), rho, D = div m^k and, on test steps, dm = m' - m.  A
// single CTA also keeps its own nodes' m and phi (and, with at most two nodes
// per thread, rho and D) in registers; in a cluster the addressing of the
// remote rows leaves no room for that without spills.  One step:
//   phase A: m' from m and phi (own, right, up; the row above the band is read
//            from the next CTA's shared memory), publish m'
//   phase B: Dn = div m' (left, below; the row below the band from the previous
//            CTA), div mbar = 2 Dn - D, phi' = phi + tau (div mbar - rho),
//            D <- Dn, publish phi'
// With C > 1 (this node-per-thread fallback) the phases are separated by
// cluster barriers (release/acquire), which also order the distributed-shared-
// memory reads of the halo rows.  The four-nodes-per-thread and wide-band
// kernels below replace those barriers by neighbour pushes: after m' a CTA
// sends its top row's m2' to the CTA above, after phi' its bottom row's phi to
// the CTA below (st.async into the neighbour's halo row, completing a
// transaction count on its mbarrier); only the boundary rows wait, with a
// bounded wait, and the CTA itself synchronises with __syncthreads.
// Stop tests: each CTA's FP64 partials go to CTA 0, which decides; every CTA
// reads the decision, so all leave the loop after the same step.

static constexpr int RES_MAX_NODES = 4096;  // nodes per CTA (512 threads x 8)
static constexpr int RES_THREADS = 1024;
static constexpr int RES_RED_BYTES = 1024;  // 32 warps x 3 doubles
static constexpr int RES_SLOT_BYTES = 512;  // 16 CTAs x 3 doubles + decision
static constexpr int RESW_RUNS = 4;         // wide bands: runs of four nodes per thread
static constexpr int RESW_MAX_NODES = RES_THREADS * 4 * RESW_RUNS;  // 16384
static constexpr int RESW_RUN_STRIDE = 4 * RES_THREADS;              // band nodes between a thread's runs
// a CTA waiting for a neighbour's halo row gives up after this long and reports
// a timeout (the neighbour is at most one step behind in a correct run)
static constexpr unsigned long long RES_HALO_WAIT_NS = 200000000ull;
// wide bands in a cluster keep two halo rows of nx floats beside the band
static constexpr int RESW_MAX_HALO_X = 4096;
// tensor-memory columns of the wide level kernel (rho, D, phi, m1 of 16 nodes per thread, 32 warps)
static constexpr uint32_t RESW_TMEM_COLS = 512;

int resident_max_nodes() { return RES_MAX_NODES; }

bool resident_fits(int nx, int ny, int cluster)
{
    if (nx < 1 || ny < 1 || nx > 65535 || cluster < 1 || cluster > 16 || ny % cluster != 0) return false;
    if (cluster & (cluster - 1)) return false;
    const long long band = (long long)(ny / cluster) * nx;
    if (band <= RES_MAX_NODES) return true;
    // wide bands (four runs of four nodes per thread) need nx % 4 == 0 and a
    // multiple of 128 nodes (so that a warp's runs are all present or all
    // absent); in a cluster the halo rows limit nx to 4096
    return nx % 4 == 0 && band <= RESW_MAX_NODES && band % 128 == 0 && (cluster == 1 || nx <= RESW_MAX_HALO_X);
}

int resident_cluster_for(int nx, int ny)
{
    // the fewest CTAs that hold at most 4096 nodes each; else the most CTAs
    // (the fastest step) with wide bands of up to 16384 nodes
    const int cs[5] = {1, 2, 4, 8, 16};
    for (int c : cs)
        if (resident_fits(nx, ny, c) && (long long)(ny / c) * nx <= RES_MAX_NODES) return c;
    for (int k = 4; k >= 0; --k)
        if (resident_fits(nx, ny, cs[k])) return cs[k];
    return 0;
}

static size_t resident_smem(int band)
{
    return RES_RED_BYTES + RES_SLOT_BYTES + (size_t)band * 7 * sizeof(float);
}

template <int NORM, int NPT, bool CL>
__global__ void __launch_bounds__(NPT >= 8 ? RES_THREADS / 2 : RES_THREADS, 1) k_resident(ResArgs a)
{
    const IterArgs& P = a.it;
    int C = 1, rank = 0;
    if (CL) {
        cg::cluster_group cl = cg::this_cluster();
        C = (int)cl.num_blocks();
        rank = (int)cl.block_rank();
    }
    const int pair = blockIdx.x / C;
    Ctl* pc = P.ctl ? P.ctl + pair : nullptr;
    if (pc && pc->error) return;  // uniform over the cluster (one pair)
    const int nx = P.nx, ny = P.ny;
    const int rows = ny / C, jb = rank * rows, nb = rows * nx;
    extern __shared__ __align__(16) unsigned char smraw[];
    double* red = reinterpret_cast<double*>(smraw);
    double* slots = reinterpret_cast<double*>(smraw + RES_RED_BYTES);  // [16][3] + decision at [48]
    float* ph = reinterpret_cast<float*>(smraw + RES_RED_BYTES + RES_SLOT_BYTES);
    float* s1 = ph + nb;
    float* s2 = s1 + nb;
    float* e1s = s2 + nb;
    float* e2s = e1s + nb;
    float* rs = e2s + nb;
    float* Ds = rs + nb;
    const size_t off = (size_t)pair * P.stride + (size_t)jb * nx;
    constexpr bool SREG = !CL;                // m and phi of own nodes in registers (single CTA)
    constexpr bool REG = SREG && NPT <= 2;    // rho and D in registers too

    const float mu = P.mu, tau = P.tau, ih = P.ih;
    const int T = blockDim.x;
    float m1r[NPT], m2r[NPT], pr[NPT], rr[REG ? NPT : 1], Dr[REG ? NPT : 1];
    int ij[NPT];  // i | (local row << 16), -1: no node
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        const int idx = threadIdx.x + k * T;
        ij[k] = -1;
        m1r[k] = m2r[k] = pr[k] = 0.f;
        if (REG) rr[REG ? k : 0] = Dr[REG ? k : 0] = 0.f;
        if (idx < nb) {
            const int jl = idx / nx, i = idx - jl * nx;
            ij[k] = i | (jl << 16);
            m1r[k] = a.m1[off + idx];
            m2r[k] = a.m2[off + idx];
            pr[k] = a.phi[off + idx];
            if (REG) rr[REG ? k : 0] = a.rho[off + idx];
            else rs[idx] = a.rho[off + idx];
            ph[idx] = pr[k];
            s1[idx] = m1r[k];
            s2[idx] = m2r[k];
        }
    }
    if (CL) cg::this_cluster().sync();
    else __syncthreads();
    // remote rows: the first row of the next CTA's phi, the last row of the
    // previous CTA's m2' (and dm2); CTA 0's decision slots
    const int last_row = (rows - 1) * nx;
    uint32_t ph_up = 0, s2_dn = 0, e2_dn = 0, slots0 = smem_u32(slots);
    if (CL) {
        if (rank + 1 < C) ph_up = dsmem_map(smem_u32(ph), rank + 1);
        if (rank > 0) {
            s2_dn = dsmem_map(smem_u32(s2 + last_row), rank - 1);
            e2_dn = dsmem_map(smem_u32(e2s + last_row), rank - 1);
        }
        slots0 = dsmem_map(smem_u32(slots), 0);
    }

    // D^0 = div m^0
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        if (ij[k] < 0) continue;
        const int idx = threadIdx.x + k * T, i = ij[k] & 0xffff, jl = ij[k] >> 16;
        const float l1 = i > 0 ? s1[idx - 1] : 0.f;
        const float d2 = jl > 0 ? s2[idx - nx] : ((CL && rank > 0) ? dsmem_ld(s2_dn + 4u * i) : 0.f);
        const float D0 = ((s1[idx] - l1) + (s2[idx] - d2)) * ih;
        if (REG) Dr[REG ? k : 0] = D0;
        else Ds[idx] = D0;
    }
    if (CL) cg::this_cluster().sync();
    else __syncthreads();

    unsigned long long t0 = 0;
    if (rank == 0 && threadIdx.x == 0) t0 = globaltimer();
    long long it = 0;
    double R = 0.0;
    int conv = 0, late = 0;
    const long long cap = P.cap;
    while (it < cap) {
        const bool check = P.fixed ? (it + 1 == cap) : ((it + 1) % P.K == 0);
        float sa = 0.f, sb = 0.f, sc = 0.f;  // FP32 terms and per-thread partials, FP64 across threads
        // ---- phase A: m' = prox(m + mu grad phi)
        auto phaseA = [&](int k) {
            const int idx = threadIdx.x + k * T, i = ij[k] & 0xffff, jl = ij[k] >> 16, j = jb + jl;
            const float pc_ = SREG ? pr[k] : ph[idx];
            const float a1 = SREG ? m1r[k] : s1[idx];
            const float a2 = SREG ? m2r[k] : s2[idx];
            float g1 = 0.f, g2 = 0.f;
            if (i < nx - 1) g1 = (ph[idx + 1] - pc_) * ih;
            if (j < ny - 1) g2 = ((jl < rows - 1 ? ph[idx + nx] : dsmem_ld(ph_up + 4u * i)) - pc_) * ih;
            float n1, n2;
            prox<NORM>(a1 + mu * g1, a2 + mu * g2, mu, n1, n2);
            if (i == nx - 1) n1 = 0.f;
            if (j == ny - 1) n2 = 0.f;
            if (check) {
                const float d1 = n1 - a1, d2 = n2 - a2;
                e1s[idx] = d1;
                e2s[idx] = d2;
                sa = fmaf(d1, d1, fmaf(d2, d2, sa));
            }
            if (SREG) {
                m1r[k] = n1;
                m2r[k] = n2;
            }
            s1[idx] = n1;
            s2[idx] = n2;
        };
        // ---- phase B: phi' = phi + tau (div(2m' - m) - rho)
        auto phaseB = [&](int k) {
            const int idx = threadIdx.x + k * T, i = ij[k] & 0xffff, jl = ij[k] >> 16;
            const float l1 = i > 0 ? s1[idx - 1] : 0.f;
            const float d2 = jl > 0 ? s2[idx - nx] : ((CL && rank > 0) ? dsmem_ld(s2_dn + 4u * i) : 0.f);
            const float o1 = SREG ? m1r[k] : s1[idx];
            const float o2 = SREG ? m2r[k] : s2[idx];
            const float pc_ = SREG ? pr[k] : ph[idx];
            const float Dn = ((o1 - l1) + (o2 - d2)) * ih;
            const float Dk = REG ? Dr[REG ? k : 0] : Ds[idx];
            const float rk = REG ? rr[REG ? k : 0] : rs[idx];
            const float pn = pc_ + tau * ((2.f * Dn - Dk) - rk);
            if (check) {
                const float el = i > 0 ? e1s[idx - 1] : 0.f;
                const float eb = jl > 0 ? e2s[idx - nx] : ((CL && rank > 0) ? dsmem_ld(e2_dn + 4u * i) : 0.f);
                const float dd = (e1s[idx] - el) + (e2s[idx] - eb);  // h div dm
                const float ep = pn - pc_;
                sb = fmaf(ep, ep, sb);
                sc = fmaf(ep, dd, sc);
            }
            if (REG) Dr[REG ? k : 0] = Dn;
            else Ds[idx] = Dn;
            if (SREG) pr[k] = pn;
            ph[idx] = pn;
        };
#pragma unroll
        for (int k = 0; k < NPT; ++k)
            if (ij[k] >= 0) phaseA(k);
        if (CL) {
            cluster_arrive();
            cluster_wait();
        } else {
            __syncthreads();
        }
#pragma unroll
        for (int k = 0; k < NPT; ++k)
            if (ij[k] >= 0) phaseB(k);
        if (CL) {
            cluster_arrive();
            cluster_wait();
        } else {
            __syncthreads();
        }
        ++it;
        if (check) {
            double v[3];
            ff_block_sum3(sa, sb, sc, reinterpret_cast<float*>(red), v);
            if (threadIdx.x == 0) {
                dsmem_st_f64(slots0 + 8u * (rank * 3 + 0), v[0]);
                dsmem_st_f64(slots0 + 8u * (rank * 3 + 1), v[1]);
                dsmem_st_f64(slots0 + 8u * (rank * 3 + 2), v[2]);
            }
            if (CL) cg::this_cluster().sync();
            else __syncthreads();
            if (rank == 0 && threadIdx.x == 0) {
                CSum t[3];
                for (int r = 0; r < C; ++r)
                    for (int c = 0; c < 3; ++c) t[c].add(slots[r * 3 + c]);
                const double Rk = (t[0].value() / (double)mu + t[1].value() / (double)tau -
                                   2.0 * (t[2].value() / P.h)) * P.h * P.h;
                const int cv = Rk < P.tol;
                const int lt = (globaltimer() - t0) > P.budget_ns;
                const int stop = P.fixed || cv || lt || it >= cap;
                slots[48] = Rk;
                slots[49] = (double)(cv | (lt << 1) | (stop << 2));
            }
            if (CL) cg::this_cluster().sync();
            else __syncthreads();
            R = dsmem_ld_f64(slots0 + 8u * 48);
            const int d = (int)dsmem_ld_f64(slots0 + 8u * 49);
            conv = d & 1;
            late = (d >> 1) & 1;
            if (d & 4) break;
        }
    }
    // write the level state back
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        if (ij[k] < 0) continue;
        const int idx = threadIdx.x + k * T;
        a.m1[off + idx] = SREG ? m1r[k] : s1[idx];
        a.m2[off + idx] = SREG ? m2r[k] : s2[idx];
        a.phi[off + idx] = SREG ? pr[k] : ph[idx];
    }
    if (rank == 0 && threadIdx.x == 0) {
        if (pc) {
            pc->iters[P.level] = it;
            pc->fpr[P.level] = R;
            pc->conv[P.level] = conv;
            if (late && !conv) pc->timeout = 1;
        }
        if (P.fpr_out) P.fpr_out[pair] = R;
        if (P.iters_out) P.iters_out[pair] = it;
    }
    // keep every CTA's shared memory alive until the remote reads are done
    if (CL) cg::this_cluster().sync();
}

// Vectorised variant for rows whose width is a multiple of 4: a thread owns
// four consecutive nodes of one row and keeps their m1, m2, phi, rho and
// D = div m^k in registers.  Shared memory holds the band's phi, m1', m2' (and
// dm on test steps) so that neighbours can read them: the row above and the
// row below as one 16-byte access, the left/right neighbour of the run as one
// scalar access.  Same arithmetic and stop test as k_resident.

// One level of one pair, on CTA `rank` of a group of C (a cluster when CL).
template <int NORM, bool CL>
__device__ __forceinline__ void res4_level(const ResArgs& a, const int pair, const int C, const int rank,
                                           unsigned char* smraw)
{
    const IterArgs& P = a.it;
    Ctl* pc = P.ctl ? P.ctl + pair : nullptr;
    if (pc && pc->error) return;  // uniform over the cluster (one pair)
    const int nx = P.nx, ny = P.ny;
    const int rows = ny / C, jb = rank * rows, nb = rows * nx;
    const int W = nx >> 2;  // threads per row
    double* red = reinterpret_cast<double*>(smraw);
    double* slots = reinterpret_cast<double*>(smraw + RES_RED_BYTES);
    float* ph = reinterpret_cast<float*>(smraw + RES_RED_BYTES + RES_SLOT_BYTES);
    float* s1 = ph + nb;
    float* s2 = s1 + nb;
    float* e1s = s2 + nb;
    float* e2s = e1s + nb;
    // cluster: phi of the row above the band (pushed by CTA rank + 1 after each
    // step) and m2' of the row below it (pushed by CTA rank - 1 after each m'),
    // with one mbarrier each in the slot area
    float* hphi = e2s + nb;
    float* hm2 = hphi + nx;
    const uint32_t bar_phi = smem_u32(slots + 56), bar_m2 = smem_u32(slots + 57);
    const size_t off = (size_t)pair * P.stride + (size_t)jb * nx;
    const float mu = P.mu, tau = P.tau;
    const float cm = P.mu * P.ih, ct = P.tau * P.ih;  // mu / h, tau / h

    const int t = threadIdx.x, lane = t & 31;
    const bool own = t < rows * W;
    const int jl = own ? t / W : 0;
    const int i0 = own ? 4 * (t - jl * W) : 0;
    const int idx = jl * nx + i0;  // = 4 t: consecutive threads own consecutive runs
    const int j = jb + jl;
    const bool last_col = own && (i0 + 4 == nx);
    const bool top = j == ny - 1;
    // own nodes: m, phi, rho and D = h div m^k, all in registers
    float m1[4] = {0.f, 0.f, 0.f, 0.f}, m2[4] = {0.f, 0.f, 0.f, 0.f}, pv[4] = {0.f, 0.f, 0.f, 0.f};
    float rv[4] = {0.f, 0.f, 0.f, 0.f}, Dv[4] = {0.f, 0.f, 0.f, 0.f};
    if (own) {
        float4 x1 = *reinterpret_cast<const float4*>(a.m1 + off + idx);
        float4 x2 = *reinterpret_cast<const float4*>(a.m2 + off + idx);
        const float4 xp = *reinterpret_cast<const float4*>(a.phi + off + idx);
        const float4 xr = *reinterpret_cast<const float4*>(a.rho + off + idx);
        // the pinned entries (zero flux through the right and top boundaries) are zero
        if (last_col) x1.w = 0.f;
        if (top) x2 = make_float4(0.f, 0.f, 0.f, 0.f);
        m1[0] = x1.x; m1[1] = x1.y; m1[2] = x1.z; m1[3] = x1.w;
        m2[0] = x2.x; m2[1] = x2.y; m2[2] = x2.z; m2[3] = x2.w;
        pv[0] = xp.x; pv[1] = xp.y; pv[2] = xp.z; pv[3] = xp.w;
        rv[0] = xr.x; rv[1] = xr.y; rv[2] = xr.z; rv[3] = xr.w;
        *reinterpret_cast<float4*>(ph + idx) = xp;
        *reinterpret_cast<float4*>(s1 + idx) = x1;
        *reinterpret_cast<float4*>(s2 + idx) = x2;
    }
    // each halo row arrives as nx floats per step; phase 0 of bar_phi is the
    // initial phi, phase s the phi after step s; phase s of bar_m2 the m2' of
    // step s + 1
    const bool has_up = CL && rank + 1 < C, has_dn = CL && rank > 0;
    const bool pushes = rank + 1 != a.drop_rank;  // false only under fault injection
    if (CL && t == 0) {
        mbar_init(bar_phi, 1);
        mbar_init(bar_m2, 1);
        if (has_up) mbar_expect(bar_phi, 4u * nx);
        if (has_dn) mbar_expect(bar_m2, 4u * nx);
        mbar_init_fence();
    }
    if (CL) cg::this_cluster().sync();
    else __syncthreads();
    const int last_row = (rows - 1) * nx;
    const bool row_top = own && jl == rows - 1, row_bot = own && jl == 0;
    const int t_top = (rows - 1) * W;  // re-arms bar_phi
    uint32_t s2_dn = 0, e2_dn = 0, slots0 = smem_u32(slots);
    if (CL) {
        if (rank > 0) {
            s2_dn = dsmem_map(smem_u32(s2 + last_row + i0), rank - 1);
            e2_dn = dsmem_map(smem_u32(e2s + last_row + i0), rank - 1);
        }
        slots0 = dsmem_map(smem_u32(slots), 0);
        // the initial phi of the bottom row goes to the CTA below
        if (row_bot && has_dn && pushes)
            st_async4(dsmem_map(smem_u32(hphi + i0), rank - 1), make_float4(pv[0], pv[1], pv[2], pv[3]),
                      dsmem_map(bar_phi, rank - 1));
    }
    unsigned par = 0;       // parity of the halo phase the next step waits for
    bool sync_fail = false;  // a halo wait ran out of time (reported as a timeout)
    auto halo_wait = [&](uint32_t bar) {
        if (!sync_fail && !mbar_wait(bar, par, RES_HALO_WAIT_NS)) {
            sync_fail = true;
            dsmem_st_f64(slots0 + 8u * 51, 1.0);
        }
    };
    // m2 of the row below the run (zero flux below the grid)
    auto below4 = [&](const float* arr, uint32_t remote) -> float4 {
        if (jl > 0) return *reinterpret_cast<const float4*>(arr + idx - nx);
        if (CL && rank > 0) return dsmem_ld4(remote);
        return make_float4(0.f, 0.f, 0.f, 0.f);
    };
    // m1 of the node left of the run: the previous lane's last node, or shared
    // memory for lane 0 (every lane takes part in the shuffle)
    auto left_of = [&](float prev_lane, const float* arr) -> float {
        if (i0 == 0) return 0.f;
        return lane == 0 ? arr[idx - 1] : prev_lane;
    };
    {  // D^0 = h div m^0
        const float ln = __shfl_up_sync(FULL, m1[3], 1);
        if (own) {
            const float l = left_of(ln, s1);
            const float4 b = below4(s2, s2_dn);
            const float bb[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int c = 0; c < 4; ++c) Dv[c] = (m1[c] - (c ? m1[c - 1] : l)) + (m2[c] - bb[c]);
        }
    }
    if (CL) cg::this_cluster().sync();
    else __syncthreads();

    // the start time, R^k and the decision live in CTA 0's slots (registers are scarce)
    if (rank == 0 && t == 0) {
        reinterpret_cast<unsigned long long*>(slots)[50] = globaltimer();
        slots[48] = 0.0;
        slots[49] = 0.0;
        slots[51] = 0.0;
    }
    if (CL) cg::this_cluster().sync();
    else __syncthreads();
    int it = 0;
    const int cap = (int)min(P.cap, (long long)INT_MAX);
    int next = P.fixed ? cap : P.K;  // step after which the next test runs
    float sa = 0.f, sb = 0.f, sc = 0.f;  // FP32 terms and per-thread partials, FP64 across threads
    // one step; the test-step work is compiled only into the step that tests
    auto one_step = [&](auto test) {
        constexpr bool check = decltype(test)::value;
        // ---- phase A: m' = prox(m + mu grad phi); on the last column and the top
        // row the gradient component is zero and so is m, hence m' too
        const float rn = __shfl_down_sync(FULL, pv[0], 1);
        if (own) {
            float up[4] = {pv[0], pv[1], pv[2], pv[3]};
            if (!top) {
                float4 u;
                if (!CL || jl < rows - 1) {
                    u = *reinterpret_cast<const float4*>(ph + idx + nx);
                } else {  // the top row of a band below another CTA's
                    halo_wait(bar_phi);
                    u = *reinterpret_cast<const float4*>(hphi + i0);
                    if (t == t_top && !sync_fail) mbar_expect(bar_phi, 4u * nx);
                }
                up[0] = u.x; up[1] = u.y; up[2] = u.z; up[3] = u.w;
            }
            const float right = last_col ? pv[3] : (lane == 31 ? ph[idx + 4] : rn);
            float n1[4], n2[4];
            if constexpr (!CL) {  // one CTA: scalar (measured faster than packed here)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float pr_ = c < 3 ? pv[c + 1] : right;
                    prox<NORM>(fmaf(cm, pr_ - pv[c], m1[c]), fmaf(cm, up[c] - pv[c], m2[c]), mu, n1[c], n2[c]);
                }
            } else {
            // two nodes per packed instruction: nodes (0, 1) and (2, 3)
#pragma unroll
            for (int c = 0; c < 4; c += 2) {
                const float2 p2 = make_float2(pv[c], pv[c + 1]);
                const float2 r2 = make_float2(pv[c + 1], c + 2 < 4 ? pv[c + 2] : right);
                const float2 v1 = __ffma2_rn(splat2(cm), sub2(r2, p2), make_float2(m1[c], m1[c + 1]));
                const float2 v2 = __ffma2_rn(splat2(cm), sub2(make_float2(up[c], up[c + 1]), p2),
                                             make_float2(m2[c], m2[c + 1]));
                float2 o1, o2;
                prox_pair<NORM>(v1, v2, mu, o1, o2);
                n1[c] = o1.x;
                n1[c + 1] = o1.y;
                n2[c] = o2.x;
                n2[c + 1] = o2.y;
            }
            }
            if constexpr (check) {
                float d1[4], d2[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    d1[c] = n1[c] - m1[c];
                    d2[c] = n2[c] - m2[c];
                    sa = fmaf(d1[c], d1[c], fmaf(d2[c], d2[c], sa));
                }
                *reinterpret_cast<float4*>(e1s + idx) = make_float4(d1[0], d1[1], d1[2], d1[3]);
                *reinterpret_cast<float4*>(e2s + idx) = make_float4(d2[0], d2[1], d2[2], d2[3]);
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                m1[c] = n1[c];
                m2[c] = n2[c];
            }
            *reinterpret_cast<float4*>(s1 + idx) = make_float4(n1[0], n1[1], n1[2], n1[3]);
            *reinterpret_cast<float4*>(s2 + idx) = make_float4(n2[0], n2[1], n2[2], n2[3]);
            if (CL && row_top && has_up && pushes)
                st_async4(dsmem_map(smem_u32(hm2 + i0), rank + 1), make_float4(n2[0], n2[1], n2[2], n2[3]),
                          dsmem_map(bar_m2, rank + 1));
        }
        if (CL && check) {  // the test step also reads dm2 of the row below from the CTA below
            cluster_arrive();
            cluster_wait();
        } else {
            __syncthreads();
        }
        // ---- phase B: phi' = phi + tau (div(2m' - m) - rho)
        const float ln = __shfl_up_sync(FULL, m1[3], 1);
        if (own) {
            const float l = left_of(ln, s1);
            float4 b;
            if (jl > 0) {
                b = *reinterpret_cast<const float4*>(s2 + idx - nx);
            } else if (has_dn) {
                halo_wait(bar_m2);
                b = *reinterpret_cast<const float4*>(hm2 + i0);
                if (t == 0 && !sync_fail) mbar_expect(bar_m2, 4u * nx);
            } else {
                b = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            const float bb[4] = {b.x, b.y, b.z, b.w};
            float pn[4];
            if constexpr (!CL) {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float Dn = (m1[c] - (c ? m1[c - 1] : l)) + (m2[c] - bb[c]);
                    pn[c] = fmaf(ct, fmaf(2.f, Dn, -Dv[c]), fmaf(-tau, rv[c], pv[c]));
                    Dv[c] = Dn;
                }
            } else {
#pragma unroll
            for (int c = 0; c < 4; c += 2) {
                const float2 Dn = __fadd2_rn(sub2(make_float2(m1[c], m1[c + 1]), make_float2(c ? m1[c - 1] : l, m1[c])),
                                             sub2(make_float2(m2[c], m2[c + 1]), make_float2(bb[c], bb[c + 1])));
                const float2 q = __ffma2_rn(splat2(ct), __ffma2_rn(splat2(2.f), Dn, neg2(make_float2(Dv[c], Dv[c + 1]))),
                                            __ffma2_rn(splat2(-tau), make_float2(rv[c], rv[c + 1]),
                                                       make_float2(pv[c], pv[c + 1])));
                pn[c] = q.x;
                pn[c + 1] = q.y;
                Dv[c] = Dn.x;
                Dv[c + 1] = Dn.y;
            }
            }
            if constexpr (check) {
                const float4 e1 = *reinterpret_cast<const float4*>(e1s + idx);
                const float4 e2 = *reinterpret_cast<const float4*>(e2s + idx);
                const float el = i0 > 0 ? e1s[idx - 1] : 0.f;
                const float4 eb = below4(e2s, e2_dn);
                const float a1[4] = {e1.x, e1.y, e1.z, e1.w}, a2[4] = {e2.x, e2.y, e2.z, e2.w};
                const float bl[4] = {eb.x, eb.y, eb.z, eb.w};
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float left = c ? a1[c - 1] : el;
                    const float dd = (a1[c] - left) + (a2[c] - bl[c]);  // h div dm
                    const float ep = pn[c] - pv[c];
                    sb = fmaf(ep, ep, sb);
                    sc = fmaf(ep, dd, sc);
                }
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) pv[c] = pn[c];
            *reinterpret_cast<float4*>(ph + idx) = make_float4(pn[0], pn[1], pn[2], pn[3]);
            if (CL && row_bot && has_dn && pushes)
                st_async4(dsmem_map(smem_u32(hphi + i0), rank - 1), make_float4(pn[0], pn[1], pn[2], pn[3]),
                          dsmem_map(bar_phi, rank - 1));
        }
        par ^= 1u;
        __syncthreads();
    };
    while (it < cap) {
        // plain steps up to the one that tests
        const int plain = (next - 1 < cap ? next - 1 : cap) - it;
        for (int r = 0; r < plain; ++r) one_step(std::false_type{});
        it += plain;
        if (it >= cap) break;
        sa = sb = sc = 0.f;
        one_step(std::true_type{});
        ++it;
        {
            next += P.K;
            double v[3];
            ff_block_sum3(sa, sb, sc, reinterpret_cast<float*>(red), v);
            if (t == 0) {
                dsmem_st_f64(slots0 + 8u * (rank * 3 + 0), v[0]);
                dsmem_st_f64(slots0 + 8u * (rank * 3 + 1), v[1]);
                dsmem_st_f64(slots0 + 8u * (rank * 3 + 2), v[2]);
            }
            if (CL) cg::this_cluster().sync();
            else __syncthreads();
            if (rank == 0 && t == 0) {
                CSum tt[3];
                for (int r = 0; r < C; ++r)
                    for (int c = 0; c < 3; ++c) tt[c].add(slots[r * 3 + c]);
                const double Rk = (tt[0].value() / (double)mu + tt[1].value() / (double)tau -
                                   2.0 * (tt[2].value() / P.h)) * P.h * P.h;
                const int cv = Rk < P.tol;
                const int lt = (globaltimer() - reinterpret_cast<const unsigned long long*>(slots)[50]) > P.budget_ns ||
                               slots[51] != 0.0;
                const int stop = P.fixed || cv || lt || it >= cap;
                slots[48] = Rk;
                slots[49] = (double)((cv && slots[51] == 0.0) | (lt << 1) | (stop << 2));
            }
            if (CL) cg::this_cluster().sync();
            else __syncthreads();
            if ((int)dsmem_ld_f64(slots0 + 8u * 49) & 4) break;
        }
    }
    // the phi pushed by the CTA above after the last step has not been read:
    // wait for it so that no copy into this CTA is in flight when it exits
    if (CL && row_top && has_up) halo_wait(bar_phi);
    if (own) {
        *reinterpret_cast<float4*>(a.m1 + off + idx) = make_float4(m1[0], m1[1], m1[2], m1[3]);
        *reinterpret_cast<float4*>(a.m2 + off + idx) = make_float4(m2[0], m2[1], m2[2], m2[3]);
        *reinterpret_cast<float4*>(a.phi + off + idx) = make_float4(pv[0], pv[1], pv[2], pv[3]);
    }
    if (rank == 0 && t == 0) {
        const double R = slots[48];
        const int d = (int)slots[49], conv = d & 1, late = (d >> 1) & 1;
        if (pc) {
            pc->iters[P.level] = it;
            pc->fpr[P.level] = R;
            pc->conv[P.level] = conv;
            if (late && !conv) pc->timeout = 1;
        }
        if (P.fpr_out) P.fpr_out[pair] = R;
        if (P.iters_out) P.iters_out[pair] = it;
    }
    if (CL) {
        cg::this_cluster().sync();  // every halo row has been consumed
        if (t == 0) {
            mbar_inval(bar_phi);
            mbar_inval(bar_m2);
        }
    }
}

template <int NORM, bool CL>
__global__ void __launch_bounds__(RES_THREADS, 1) k_resident4(ResArgs a)
{
    int C = 1, rank = 0;
    if (CL) {
        cg::cluster_group cl = cg::this_cluster();
        C = (int)cl.num_blocks();
        rank = (int)cl.block_rank();
    }
    extern __shared__ __align__(16) unsigned char smraw[];
    res4_level<NORM, CL>(a, blockIdx.x / C, C, rank, smraw);
}

// Wide-band variant for levels of up to 16 x 16384 nodes (512 x 512 in one
// 16-CTA cluster): a thread owns four runs of four nodes.  Shared memory holds
// phi, m1 and m2 of the band (12 B per node, 192 KB at 16384 nodes) and two
// halo rows for the neighbours; each thread's own rho, D = h div m^k, phi and
// m1 live in tensor memory (wide_level with TM; without it, own values are
// re-read from shared memory, rho from L1/L2, and D stays in registers).  The
// test step's cross term
// <dphi, div dm> uses div dm = div m' - div m^k, both already formed in FP32
// (no shared-memory copy of dm is needed).

static size_t resident_wide_smem(int band)
{
    // + the two halo rows of a cluster band (at most RESW_MAX_HALO_X wide)
    return RES_RED_BYTES + RES_SLOT_BYTES + (size_t)band * 3 * sizeof(float) + 2 * RESW_MAX_HALO_X * sizeof(float);
}

// TM: the thread's own rho, D = h div m^k, phi and m1 live in tensor memory
// (16 columns per run, 64 per warp, all 512 of the SM): rho is not re-read from
// L2 every step (shared memory is full with the band), D leaves the registers,
// and shared memory serves only what neighbours read (phi, m2, and the last
// m1 of each run)
template <int NORM, bool CL, bool TM = false>
__device__ __forceinline__ void wide_level(const ResArgs& a, const int pair, const int C, const int rank,
                                           unsigned char* smraw)
{
    const IterArgs& P = a.it;
    auto group_sync = [&]() {
        if (CL) cg::this_cluster().sync();
        else __syncthreads();
    };
    Ctl* pc = P.ctl ? P.ctl + pair : nullptr;
    if (pc && pc->error) return;  // uniform over the cluster (one pair)
    const int nx = P.nx, ny = P.ny;
    const int rows = ny / C, jb = rank * rows, nb = rows * nx;
    double* red = reinterpret_cast<double*>(smraw);
    double* slots = reinterpret_cast<double*>(smraw + RES_RED_BYTES);
    float* ph = reinterpret_cast<float*>(smraw + RES_RED_BYTES + RES_SLOT_BYTES);
    float* s1 = ph + nb;
    float* s2 = s1 + nb;
    // cluster halo rows and their mbarriers (the exchange of res4_level)
    float* hphi = s2 + nb;
    float* hm2 = hphi + nx;
    const uint32_t bar_phi = smem_u32(slots + 56), bar_m2 = smem_u32(slots + 57);
    const bool has_up = CL && rank + 1 < C, has_dn = CL && rank > 0;
    const bool pushes = rank + 1 != a.drop_rank;  // false only under fault injection
    const size_t off = (size_t)pair * P.stride + (size_t)jb * nx;
    const float mu = P.mu, tau = P.tau;
    const float cm = P.mu * P.ih, ct = P.tau * P.ih;  // mu / h, tau / h
    const int t = threadIdx.x, T = blockDim.x, lane = t & 31;
    // tensor memory: warp w uses lanes 32 (w % 4) .. + 31 and columns 16 (w / 4) .. + 15
    uint32_t tb = 0;
    if (TM) {
        if (t < 32) {
            // no relinquish_alloc_permit: the persistent cascade allocates again
            // for every wide level it runs (one CTA per SM, nothing else competes)
            tmem_alloc(smem_u32(slots + 58), RESW_TMEM_COLS);
        }
        tmem_fence_before();
        __syncthreads();
        tmem_fence_after();
        tb = *reinterpret_cast<volatile uint32_t*>(slots + 58) + ((32u * ((t >> 5) & 3)) << 16) +
             64u * (uint32_t)(t >> 7);
    }
    // run r of this thread: nodes 4 q .. 4 q + 3 of the band, q = t + r T;
    // pk = (row << 16) | column of its first node, or -1 past the band
    int pk[RESW_RUNS];
    // the band index of run r's first node is id0 + r RESW_RUN_STRIDE (blockDim.x == RES_THREADS)
    const int id0 = 4 * t;
    // h div m^k in registers unless it lives in tensor memory (then rho is there
    // too; otherwise rho is re-read from L1/L2 every step: registers are scarce)
    float Dv[TM ? 1 : RESW_RUNS][4];
    const float* __restrict__ rho = a.rho + off;
#pragma unroll
    for (int r = 0; r < RESW_RUNS; ++r) {
        const int id = 4 * (t + r * T);
        pk[r] = -1;
        if (id < nb) {
            const int jl = id / nx, i0 = id - jl * nx;
            pk[r] = (jl << 16) | i0;
            float4 x1 = *reinterpret_cast<const float4*>(a.m1 + off + id);
            float4 x2 = *reinterpret_cast<const float4*>(a.m2 + off + id);
            const float4 xp = *reinterpret_cast<const float4*>(a.phi + off + id);
            // the pinned entries (zero flux through the right and top boundaries) are zero
            if (i0 + 4 == nx) x1.w = 0.f;
            if (jb + jl == ny - 1) x2 = make_float4(0.f, 0.f, 0.f, 0.f);
            *reinterpret_cast<float4*>(ph + id) = xp;
            *reinterpret_cast<float4*>(s1 + id) = x1;
            *reinterpret_cast<float4*>(s2 + id) = x2;
            if (TM) {
                tmem_st4(tb + 16u * r, __ldg(reinterpret_cast<const float4*>(rho + id)));
                tmem_st4(tb + 16u * r + 8u, xp);
                tmem_st4(tb + 16u * r + 12u, x1);
            }
        }
    }
    if (TM) tmem_wait_st();
    if (CL && t == 0) {
        mbar_init(bar_phi, 1);
        mbar_init(bar_m2, 1);
        if (has_up) mbar_expect(bar_phi, 4u * nx);
        if (has_dn) mbar_expect(bar_m2, 4u * nx);
        mbar_init_fence();
    }
    group_sync();
    const int last_row = (rows - 1) * nx;
    const int t_top = (last_row >> 2) % T;  // owns the first run of the top row: re-arms bar_phi
    uint32_t s2_dn = 0u, slots0 = smem_u32(slots);
    if (CL) {
        if (rank > 0) s2_dn = dsmem_map(smem_u32(s2 + last_row), rank - 1);
        slots0 = dsmem_map(smem_u32(slots), 0);
    }
    unsigned par = 0;        // parity of the halo phase the next step waits for
    bool sync_fail = false;  // a halo wait ran out of time (reported as a timeout)
    auto halo_wait = [&](uint32_t bar) {
        if (!sync_fail && !mbar_wait(bar, par, RES_HALO_WAIT_NS)) {
            sync_fail = true;
            dsmem_st_f64(slots0 + 8u * 51, 1.0);
        }
    };
    // h div of the m currently in s1, s2 at run r (the left neighbour comes from the
    // previous lane by a shuffle: a warp's runs are all present or all absent,
    // since the band holds a multiple of 128 nodes); the row below the band is
    // read from the CTA below (initial state) or from the halo row it pushed
    // m1 of the run: given by the caller (tm1, loaded from tensor memory with the
    // run's other values), else read from shared memory
    auto divergence = [&](auto rc, float out[4], auto halo, const float4* tm1) {
        constexpr int r = decltype(rc)::value;
        const int jl = pk[r] >> 16, i0 = pk[r] & 0xffff, id = id0 + r * RESW_RUN_STRIDE;
        const float4 m1 = tm1 ? *tm1 : *reinterpret_cast<const float4*>(s1 + id);
        const float ln = __shfl_up_sync(FULL, m1.w, 1);
        const float4 m2 = *reinterpret_cast<const float4*>(s2 + id);
        const float l = i0 == 0 ? 0.f : (lane == 0 ? s1[id - 1] : ln);
        float4 b = make_float4(0.f, 0.f, 0.f, 0.f);
        if (jl > 0) {
            b = *reinterpret_cast<const float4*>(s2 + id - nx);
        } else if (has_dn) {
            if constexpr (decltype(halo)::value) {
                halo_wait(bar_m2);
                b = *reinterpret_cast<const float4*>(hm2 + i0);
                if (t == 0 && r == 0 && !sync_fail) mbar_expect(bar_m2, 4u * nx);
            } else {
                b = dsmem_ld4(s2_dn + 4u * i0);
            }
        }
        const float2 d01 = __fadd2_rn(sub2(make_float2(m1.x, m1.y), make_float2(l, m1.x)),
                                      sub2(make_float2(m2.x, m2.y), make_float2(b.x, b.y)));
        const float2 d23 = __fadd2_rn(sub2(make_float2(m1.z, m1.w), make_float2(m1.y, m1.z)),
                                      sub2(make_float2(m2.z, m2.w), make_float2(b.z, b.w)));
        out[0] = d01.x;
        out[1] = d01.y;
        out[2] = d23.x;
        out[3] = d23.y;
    };
    static_for<RESW_RUNS>([&](auto rc) {
        constexpr int r = decltype(rc)::value;
        if (pk[r] >= 0) {
            if constexpr (TM) {
                float d0[4];
                divergence(rc, d0, std::false_type{}, nullptr);
                tmem_st4_at<16 * r + 4>(tb, make_float4(d0[0], d0[1], d0[2], d0[3]));
            } else {
                divergence(rc, Dv[r], std::false_type{}, nullptr);
            }
        }
    });
    if (TM) tmem_wait_st();
    // the start time, R^k and the decision live in CTA 0's slots (registers are scarce)
    if (rank == 0 && t == 0) {
        reinterpret_cast<unsigned long long*>(slots)[50] = globaltimer();
        slots[48] = 0.0;
        slots[49] = 0.0;
        slots[51] = 0.0;
    }
    group_sync();
    // the initial phi of the bottom row goes to the CTA below
    if (has_dn && pushes) {
#pragma unroll
        for (int r = 0; r < RESW_RUNS; ++r)
            if (pk[r] >= 0 && (pk[r] >> 16) == 0) {
                const int i0 = pk[r] & 0xffff;
                st_async4(dsmem_map(smem_u32(hphi + i0), rank - 1), *reinterpret_cast<const float4*>(ph + i0),
                          dsmem_map(bar_phi, rank - 1));
            }
    }
    // (a 32-bit step counter with a running "next test" step made this loop
    // several times slower here, measured; the 64-bit modulo costs little per node)
    long long it = 0;
    const long long cap = P.cap;
    float sa = 0.f, sb = 0.f, sc = 0.f;  // FP32 terms and per-thread partials, FP64 across threads
    // one step; the test-step sums are compiled only into the step that tests
    auto wstep = [&](auto test) {
        constexpr bool check = decltype(test)::value;
        // ---- phase A: m' = prox(m + mu grad phi); on the last column and the top
        // row the gradient component is zero and so is m, hence m' too
        static_for<RESW_RUNS>([&](auto rc) {
            constexpr int r = decltype(rc)::value;
            if (pk[r] < 0) return;
            const int jl = pk[r] >> 16, i0 = pk[r] & 0xffff, id = id0 + r * RESW_RUN_STRIDE;
            float4 p4, a1;  // the run's phi and m1: two loads behind one wait
            if constexpr (TM) {
                tmem_ld4x2_at<16 * r + 8, 16 * r + 12>(tb, p4, a1);
            } else {
                p4 = *reinterpret_cast<const float4*>(ph + id);
                a1 = *reinterpret_cast<const float4*>(s1 + id);
            }
            const float rn = __shfl_down_sync(FULL, p4.x, 1);
            const int j = jb + jl;
            const bool last_col = i0 + 4 == nx;
            const float4 a2 = *reinterpret_cast<const float4*>(s2 + id);
            float4 u = p4;
            if (j < ny - 1) {
                if (!CL || jl < rows - 1) {
                    u = *reinterpret_cast<const float4*>(ph + id + nx);
                } else {
                    halo_wait(bar_phi);
                    u = *reinterpret_cast<const float4*>(hphi + i0);
                    if (t == t_top && id == last_row && !sync_fail) mbar_expect(bar_phi, 4u * nx);
                }
            }
            const float right = last_col ? p4.w : (lane == 31 ? ph[id + 4] : rn);
            const float pv[4] = {p4.x, p4.y, p4.z, p4.w}, up[4] = {u.x, u.y, u.z, u.w};
            const float m1[4] = {a1.x, a1.y, a1.z, a1.w}, m2[4] = {a2.x, a2.y, a2.z, a2.w};
            float n1[4], n2[4];
#pragma unroll
            for (int c = 0; c < 4; c += 2) {  // two nodes per packed instruction
                const float2 p2 = make_float2(pv[c], pv[c + 1]);
                const float2 r2 = make_float2(pv[c + 1], c + 2 < 4 ? pv[c + 2] : right);
                const float2 v1 = __ffma2_rn(splat2(cm), sub2(r2, p2), make_float2(m1[c], m1[c + 1]));
                const float2 v2 = __ffma2_rn(splat2(cm), sub2(make_float2(up[c], up[c + 1]), p2),
                                             make_float2(m2[c], m2[c + 1]));
                float2 o1, o2;
                prox_pair<NORM>(v1, v2, mu, o1, o2);
                n1[c] = o1.x;
                n1[c + 1] = o1.y;
                n2[c] = o2.x;
                n2[c + 1] = o2.y;
            }
            if (check) {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float d1 = n1[c] - m1[c], d2 = n2[c] - m2[c];
                    sa = fmaf(d1, d1, fmaf(d2, d2, sa));
                }
            }
            if constexpr (TM) {  // neighbours read only the run's last m1 (left of the next run)
                tmem_st4_at<16 * r + 12>(tb, make_float4(n1[0], n1[1], n1[2], n1[3]));
                s1[id + 3] = n1[3];
            } else {
                *reinterpret_cast<float4*>(s1 + id) = make_float4(n1[0], n1[1], n1[2], n1[3]);
            }
            *reinterpret_cast<float4*>(s2 + id) = make_float4(n2[0], n2[1], n2[2], n2[3]);
            if (has_up && jl == rows - 1 && pushes)
                st_async4(dsmem_map(smem_u32(hm2 + i0), rank + 1), make_float4(n2[0], n2[1], n2[2], n2[3]),
                          dsmem_map(bar_m2, rank + 1));
        });
        if constexpr (TM) tmem_wait_st();  // m1' is in place before phase B reads it
        __syncthreads();
        // ---- phase B: phi' = phi + tau (div(2m' - m) - rho)
        static_for<RESW_RUNS>([&](auto rc) {
            constexpr int r = decltype(rc)::value;
            if (pk[r] < 0) return;
            float Dn[4];
            const int id = id0 + r * RESW_RUN_STRIDE;
            float4 p4, r4, d4;
            if constexpr (TM) {
                float4 m1v;  // the run's m1', phi, rho and D: four loads behind one wait
                tmem_ld4x4_at<16 * r + 12, 16 * r + 8, 16 * r, 16 * r + 4>(tb, m1v, p4, r4, d4);
                divergence(rc, Dn, std::true_type{}, &m1v);
            } else {
                divergence(rc, Dn, std::true_type{}, nullptr);
                p4 = *reinterpret_cast<const float4*>(ph + id);
                r4 = __ldg(reinterpret_cast<const float4*>(rho + id));
                d4 = make_float4(Dv[r][0], Dv[r][1], Dv[r][2], Dv[r][3]);
            }
            const float pv[4] = {p4.x, p4.y, p4.z, p4.w}, rv[4] = {r4.x, r4.y, r4.z, r4.w};
            const float Do[4] = {d4.x, d4.y, d4.z, d4.w};
            float pn[4];
#pragma unroll
            for (int c = 0; c < 4; c += 2) {
                const float2 q = __ffma2_rn(
                    splat2(ct), __ffma2_rn(splat2(2.f), make_float2(Dn[c], Dn[c + 1]), neg2(make_float2(Do[c], Do[c + 1]))),
                    __ffma2_rn(splat2(-tau), make_float2(rv[c], rv[c + 1]), make_float2(pv[c], pv[c + 1])));
                pn[c] = q.x;
                pn[c + 1] = q.y;
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                if (check) {
                    const float ep = pn[c] - pv[c];
                    sb = fmaf(ep, ep, sb);
                    sc = fmaf(ep, Dn[c] - Do[c], sc);  // h <dphi, div dm>, scaled below
                }
                if constexpr (!TM) Dv[r][c] = Dn[c];
            }
            if constexpr (TM) {
                tmem_st4_at<16 * r + 4>(tb, make_float4(Dn[0], Dn[1], Dn[2], Dn[3]));
                tmem_st4_at<16 * r + 8>(tb, make_float4(pn[0], pn[1], pn[2], pn[3]));
            }
            *reinterpret_cast<float4*>(ph + id) = make_float4(pn[0], pn[1], pn[2], pn[3]);
            if (has_dn && id < nx && pushes)
                st_async4(dsmem_map(smem_u32(hphi + id), rank - 1), make_float4(pn[0], pn[1], pn[2], pn[3]),
                          dsmem_map(bar_phi, rank - 1));
        });
        if constexpr (TM) tmem_wait_st();  // this step's D and phi are in place before the next reads them
        par ^= 1u;
        __syncthreads();
    };
    while (it < cap) {
        const bool check = P.fixed ? (it + 1 == cap) : ((it + 1) % P.K == 0);
        if (!check) {
            wstep(std::false_type{});
            ++it;
            continue;
        }
        sa = sb = sc = 0.f;
        wstep(std::true_type{});
        ++it;
        {
            double v[3];
            ff_block_sum3(sa, sb, sc, reinterpret_cast<float*>(red), v);
            if (t == 0) {
                dsmem_st_f64(slots0 + 8u * (rank * 3 + 0), v[0]);
                dsmem_st_f64(slots0 + 8u * (rank * 3 + 1), v[1]);
                dsmem_st_f64(slots0 + 8u * (rank * 3 + 2), v[2]);
            }
            group_sync();
            if (rank == 0 && t == 0) {
                CSum tt[3];
                for (int q = 0; q < C; ++q)
                    for (int c = 0; c < 3; ++c) tt[c].add(slots[q * 3 + c]);
                const double Rk = (tt[0].value() / (double)mu + tt[1].value() / (double)tau -
                                   2.0 * (tt[2].value() / P.h)) * P.h * P.h;
                const int cv = Rk < P.tol;
                const int lt = (globaltimer() - reinterpret_cast<const unsigned long long*>(slots)[50]) > P.budget_ns ||
                               slots[51] != 0.0;
                const int stop = P.fixed || cv || lt || it >= cap;
                slots[48] = Rk;
                slots[49] = (double)((cv && slots[51] == 0.0) | (lt << 1) | (stop << 2));
            }
            group_sync();
            if ((int)dsmem_ld_f64(slots0 + 8u * 49) & 4) break;
        }
    }
    // wait for the phi pushed by the CTA above after the last step (no copy
    // into this CTA may be in flight when it exits)
    if (has_up) {
        bool top_run = false;
#pragma unroll
        for (int r = 0; r < RESW_RUNS; ++r) top_run |= pk[r] >= 0 && (pk[r] >> 16) == rows - 1;
        if (top_run) halo_wait(bar_phi);
    }
#pragma unroll
    for (int r = 0; r < RESW_RUNS; ++r) {
        if (pk[r] < 0) continue;
        const int id = (pk[r] >> 16) * nx + (pk[r] & 0xffff);
        *reinterpret_cast<float4*>(a.m1 + off + id) =
            TM ? tmem_ld4(tb + 16u * r + 12u) : *reinterpret_cast<const float4*>(s1 + id);
        *reinterpret_cast<float4*>(a.m2 + off + id) = *reinterpret_cast<const float4*>(s2 + id);
        *reinterpret_cast<float4*>(a.phi + off + id) = *reinterpret_cast<const float4*>(ph + id);
    }
    if (TM) {  // every tensor-memory load has completed (each waited for its own)
        tmem_fence_before();
        __syncthreads();
        tmem_fence_after();
        if (t < 32) tmem_dealloc(*reinterpret_cast<volatile uint32_t*>(slots + 58), RESW_TMEM_COLS);
    }
    if (rank == 0 && t == 0) {
        const double R = slots[48];
        const int d = (int)slots[49], conv = d & 1, late = (d >> 1) & 1;
        if (pc) {
            pc->iters[P.level] = it;
            pc->fpr[P.level] = R;
            pc->conv[P.level] = conv;
            if (late && !conv) pc->timeout = 1;
        }
        if (P.fpr_out) P.fpr_out[pair] = R;
        if (P.iters_out) P.iters_out[pair] = it;
    }
    if (CL) {
        cg::this_cluster().sync();  // every halo row has been consumed
        if (t == 0) {
            mbar_inval(bar_phi);
            mbar_inval(bar_m2);
        }
    }
}

template <int NORM, bool CL>
__global__ void __launch_bounds__(RES_THREADS, 1) k_resident_wide(ResArgs a)
{
    int C = 1, rank = 0;
    if (CL) {
        cg::cluster_group cl = cg::this_cluster();
        C = (int)cl.num_blocks();
        rank = (int)cl.block_rank();
    }
    extern __shared__ __align__(16) unsigned char smraw[];
    wide_level<NORM, CL, true>(a, blockIdx.x / C, C, rank, smraw);
}

// ---------------------------------------------------------------------------
// Persistent cascade for mixed-size batches (one CTA per pair, every level)
// ---------------------------------------------------------------------------

int cascade_level_fits(int nx, int ny)
{
    const long long n = (long long)nx * ny;
    if (nx < 4 || ny < 1 || nx % 4 != 0 || nx > 65535) return 0;
    return (n <= RES_MAX_NODES ? 1 : 0) | ((n <= RESW_MAX_NODES && n % 128 == 0) ? 2 : 0);
}

// WIDE = false: every level on the four-nodes-per-thread layout (at most 4096
// nodes), its body inlined.  WIDE = true: levels of up to 4096 nodes on that
// layout, larger ones on the wide layout (at most 16384 nodes, a multiple of
// 128); the two bodies are separate functions here, since inlined side by side
// they spill (measured: the split is faster than the wide layout for every level).
template <int NORM>
__device__ __noinline__ void cascade_level_small(const ResArgs& a, int pair, unsigned char* smraw)
{
    res4_level<NORM, false>(a, pair, 1, 0, smraw);
}
template <int NORM>
__device__ __noinline__ void cascade_level_wide(const ResArgs& a, int pair, unsigned char* smraw)
{
    wide_level<NORM, false, true>(a, pair, 1, 0, smraw);
}

template <int NORM, bool WIDE>
__global__ void __launch_bounds__(RES_THREADS, 1) k_cascade(CascadeArgs a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    // the pair and level being solved and the level's arguments live in shared
    // memory and are re-read after every level solve: nothing but the solve's own
    // state stays in registers across it (registers are scarce at 1024 threads)
    __shared__ int s_c, s_b, s_l, s_go;
    __shared__ ResArgs s_args;
    volatile int* vc = &s_c;
    volatile int* vb = &s_b;
    volatile int* vl = &s_l;
    volatile int* vgo = &s_go;
    for (;;) {
        __syncthreads();  // the previous pair is finished before the shared fields change
        if (threadIdx.x == 0) {
            const int w = (int)atomicAdd(a.next, 1u);
            int c = 0, b = w;
            while (c < a.n_classes - 1 && b >= a.cls[c].count) {
                b -= a.cls[c].count;
                ++c;
            }
            *vc = c;
            *vb = b;
            *vl = w >= a.total ? 0 : a.cls[c].split;  // the coarse launch did the levels before
            // 0: no work left; 1: solve; 2: skip (rejected input or unused slot)
            *vgo = w >= a.total ? 0 : (a.cls[c].ctl[b].error ? 2 : 1);
        }
        __syncthreads();
        const int go = *vgo;
        if (go == 0) return;
        if (go == 2) continue;
        for (;;) {
            const int l = *vl;
            const CascadeClass* K = a.cls + *vc;
            if (l >= K->levels) break;
            const int b = *vb;
            const CascadeLevel& v = K->lv[l];
            const int n = v.nx * v.ny;
            const size_t off = (size_t)b * n;
            if (l == 0) {  // Algorithm 3 starts from m = 0, phi = 0 on the coarsest grid
                for (int k = threadIdx.x; k < n; k += blockDim.x) {
                    v.m1[off + k] = 0.f;
                    v.m2[off + k] = 0.f;
                    v.phi[off + k] = 0.f;
                }
            } else {
                const CascadeLevel& cv = K->lv[l - 1];
                const size_t co = (size_t)b * cv.nx * cv.ny;
                for (int k = threadIdx.x; k < n; k += blockDim.x) {
                    const int j = k / v.nx, i = k - j * v.nx;
                    prolong_node(cv.nx, cv.ny, cv.m1 + co, cv.m2 + co, cv.phi + co, v.m1 + off, v.m2 + off,
                                 v.phi + off, i, j);
                }
            }
            if (threadIdx.x == 0) {
                ResArgs& r = s_args;
                r = ResArgs{};
                r.m1 = v.m1;
                r.m2 = v.m2;
                r.phi = v.phi;
                r.rho = v.rho;
                r.pairs = 1;
                IterArgs& it = r.it;
                it.nx = v.nx;
                it.ny = v.ny;
                it.mu = v.mu;
                it.tau = v.tau;
                it.ih = v.ih;
                it.h = v.h;
                it.tol = v.tol;
                it.cap = a.cap;
                it.K = a.K;
                it.fixed = 0;
                it.level = l;
                it.budget_ns = a.budget_ns;
                it.stride = n;
                it.ctl = K->ctl;
            }
            __syncthreads();  // the level's state is in global memory for the level solve to load
            if (!WIDE) res4_level<NORM, false>(s_args, b, 1, 0, smraw);
            else if (n <= RES_MAX_NODES) cascade_level_small<NORM>(s_args, b, smraw);
            else cascade_level_wide<NORM>(s_args, b, smraw);
            __syncthreads();  // the level's final state is stored before the next level reads it
            if (threadIdx.x == 0) *vl = l + 1;
            __syncthreads();
        }
    }
}

// Levels of the pairs of cluster classes, in row bands over the cluster's CTAs
// (bodies kept apart from the single-CTA ones, as those are, for registers).
template <int NORM>
__device__ __noinline__ void cascade_level_split4(const ResArgs& a, int pair, int rank, unsigned char* smraw)
{
    res4_level<NORM, true>(a, pair, CASCADE_CLUSTER, rank, smraw);
}
template <int NORM>
__device__ __noinline__ void cascade_level_splitw(const ResArgs& a, int pair, int rank, unsigned char* smraw)
{
    wide_level<NORM, true, true>(a, pair, CASCADE_CLUSTER, rank, smraw);
}

// Levels that fit the four-nodes-per-thread layout of one CTA stay on CTA 0
// (split four ways they would not step faster); larger ones split into row
// bands of at least two rows when they can, else stay on CTA 0 in the wide
// layout.
int cascade_level_mode_cluster(int nx, int ny)
{
    const int f = cascade_level_fits(nx, ny);
    if (f & 1) return CASCADE_ONE4;
    if (ny / CASCADE_CLUSTER >= 2 && resident_fits(nx, ny, CASCADE_CLUSTER))
        return (long long)(ny / CASCADE_CLUSTER) * nx <= RES_MAX_NODES ? CASCADE_SPLIT4 : CASCADE_SPLITW;
    return (f & 2) ? CASCADE_ONEW : 0;
}

// The level's ResArgs for pair b of class K (thread 0 writes, the block reads
// after a barrier).
__device__ void cascade_args(ResArgs& r, const CascadeArgs& a, const CascadeClass* K, int l)
{
    const CascadeLevel& v = K->lv[l];
    r = ResArgs{};
    r.m1 = v.m1;
    r.m2 = v.m2;
    r.phi = v.phi;
    r.rho = v.rho;
    r.pairs = 1;
    IterArgs& it = r.it;
    it.nx = v.nx;
    it.ny = v.ny;
    it.mu = v.mu;
    it.tau = v.tau;
    it.ih = v.ih;
    it.h = v.h;
    it.tol = v.tol;
    it.cap = a.cap;
    it.K = a.K;
    it.fixed = 0;
    it.level = l;
    it.budget_ns = a.budget_ns;
    it.stride = v.nx * v.ny;
    it.ctl = K->ctl;
}

// Level l's starting state of pair b, nodes [k0, k1): zero on the coarsest
// level (Algorithm 3 starts from m = 0, phi = 0), else Interpolate of level l - 1.
__device__ void cascade_init(const CascadeClass* K, int l, int b, int k0, int k1)
{
    const CascadeLevel& v = K->lv[l];
    const size_t off = (size_t)b * v.nx * v.ny;
    if (l == 0) {
        for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
            v.m1[off + k] = 0.f;
            v.m2[off + k] = 0.f;
            v.phi[off + k] = 0.f;
        }
    } else {
        const CascadeLevel& cv = K->lv[l - 1];
        const size_t co = (size_t)b * cv.nx * cv.ny;
        for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
            const int j = k / v.nx, i = k - j * v.nx;
            prolong_node(cv.nx, cv.ny, cv.m1 + co, cv.m2 + co, cv.phi + co, v.m1 + off, v.m2 + off, v.phi + off, i,
                         j);
        }
    }
}

// Persistent launch in clusters of CASCADE_CLUSTER CTAs.  Phase 1: a cluster
// takes the next pair of the cluster classes (largest grids; CTA 0 draws it
// and writes it into every CTA's shared memory), initialises each level in row
// bands and solves it in row bands over the cluster (or on CTA 0 alone when
// the level cannot be split).  Phase 2, once those pairs are all taken: each
// CTA takes pairs of the single-CTA classes alone, as k_cascade does, with no
// cluster barrier and no distributed shared memory, so CTAs may leave at
// different times.
template <int NORM>
__global__ void __launch_bounds__(RES_THREADS, 1) k_cascade_cl(CascadeArgs a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ int s_c, s_b, s_l, s_go;
    __shared__ unsigned s_w;
    __shared__ ResArgs s_args;
    volatile int* vc = &s_c;
    volatile int* vb = &s_b;
    volatile int* vl = &s_l;
    volatile int* vgo = &s_go;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    for (;;) {
        cl.sync();  // every CTA has read the previous draw
        if (rank == 0 && threadIdx.x == 0) {
            const unsigned w = atomicAdd(a.next_big, 1u);
            for (int r = 0; r < CASCADE_CLUSTER; ++r) dsmem_st_u32(dsmem_map(smem_u32(&s_w), (uint32_t)r), w);
        }
        cl.sync();
        const int w = (int)*reinterpret_cast<volatile unsigned*>(&s_w);
        if (w >= a.total_big) break;  // the same draw in every CTA of the cluster
        int c = 0, b = w;
        while (c < a.n_big - 1 && b >= a.big[c].count) {
            b -= a.big[c].count;
            ++c;
        }
        const CascadeClass* K = a.big + c;
        if (K->ctl[b].error) continue;  // set before the launch: the same in every CTA
        for (int l = K->split; l < K->levels; ++l) {  // the coarse launch did the levels before
            const CascadeLevel& v = K->lv[l];
            const int rows = v.ny / CASCADE_CLUSTER, rest = v.ny - rows * CASCADE_CLUSTER;
            // row bands (the last one takes the rows a split leaves over)
            const int j0 = rank * rows, j1 = rank == CASCADE_CLUSTER - 1 ? j0 + rows + rest : j0 + rows;
            cascade_init(K, l, b, j0 * v.nx, j1 * v.nx);
            if (threadIdx.x == 0) cascade_args(s_args, a, K, l);
            cl.sync();  // the level's starting state (all bands) is in global memory
            const int mode = v.mode;
            if (mode == CASCADE_SPLIT4) cascade_level_split4<NORM>(s_args, b, rank, smraw);
            else if (mode == CASCADE_SPLITW) cascade_level_splitw<NORM>(s_args, b, rank, smraw);
            else if (rank == 0 && mode == CASCADE_ONE4) cascade_level_small<NORM>(s_args, b, smraw);
            else if (rank == 0) cascade_level_wide<NORM>(s_args, b, smraw);
            cl.sync();  // the level's final state is stored before the next level reads it
        }
    }
    // phase 2: single-CTA classes, one pair per CTA
    for (;;) {
        __syncthreads();  // the previous pair is finished before the shared fields change
        if (threadIdx.x == 0) {
            const int w = (int)atomicAdd(a.next, 1u);
            int c = 0, b = w;
            while (c < a.n_classes - 1 && b >= a.cls[c].count) {
                b -= a.cls[c].count;
                ++c;
            }
            *vc = c;
            *vb = b;
            *vl = w >= a.total ? 0 : a.cls[c].split;
            *vgo = w >= a.total ? 0 : (a.cls[c].ctl[b].error ? 2 : 1);
        }
        __syncthreads();
        const int go = *vgo;
        if (go == 0) return;
        if (go == 2) continue;
        for (;;) {
            const int l = *vl;
            const CascadeClass* K = a.cls + *vc;
            if (l >= K->levels) break;
            const int b = *vb;
            const CascadeLevel& v = K->lv[l];
            const int n = v.nx * v.ny;
            cascade_init(K, l, b, 0, n);
            if (threadIdx.x == 0) cascade_args(s_args, a, K, l);
            __syncthreads();  // the level's state is in global memory for the level solve to load
            if (n <= RES_MAX_NODES) cascade_level_small<NORM>(s_args, b, smraw);
            else cascade_level_wide<NORM>(s_args, b, smraw);
            __syncthreads();  // the level's final state is stored before the next level reads it
            if (threadIdx.x == 0) *vl = l + 1;
            __syncthreads();
        }
    }
}

static size_t cascade_smem(bool wide) { return wide ? resident_wide_smem(RESW_MAX_NODES) : resident_smem(RES_MAX_NODES); }

static const void* cascade_cl_fn(int norm)
{
    return norm == W1_NORM_L1 ? (const void*)k_cascade_cl<W1_NORM_L1>
           : norm == W1_NORM_L2 ? (const void*)k_cascade_cl<W1_NORM_L2>
                                : (const void*)k_cascade_cl<W1_NORM_LINF>;
}

static cudaLaunchConfig_t cascade_cl_config(int clusters, cudaLaunchAttribute* attr)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(clusters * CASCADE_CLUSTER, 1, 1);
    cfg.blockDim = dim3(RES_THREADS, 1, 1);
    cfg.dynamicSmemBytes = cascade_smem(true);
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CASCADE_CLUSTER;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

int cascade_clusters(int norm)
{
    cudaLaunchAttribute attr[1];
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg = cascade_cl_config(sms / CASCADE_CLUSTER, attr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, cascade_cl_fn(norm), &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

cudaError_t launch_cascade_cluster(int norm, const CascadeArgs& a, int clusters, cudaStream_t s)
{
    if (clusters < 1 || a.total + a.total_big < 1) return cudaErrorInvalidValue;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cascade_cl_config(clusters, attr);
    cfg.stream = s;
    void* args[1] = {(void*)&a};
    return cudaLaunchKernelExC(&cfg, cascade_cl_fn(norm), args);
}

// The coarse levels of every pair of a persistent launch (at most
// CASCADE_COARSE_NODES nodes each: 16^2 and 32^2 for the usual cascades).  The
// persistent CTA has 1024 threads and the whole SM; a 16^2 level keeps 64 of
// them busy for thousands of steps.  Here a CTA of CASCADE_COARSE_THREADS takes
// a pair and runs its coarse levels, several CTAs to an SM; the persistent
// launch that follows continues every pair from its first larger level.
template <int NORM>
__global__ void __launch_bounds__(CASCADE_COARSE_THREADS, 3) k_cascade_coarse(CascadeArgs a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ int s_c, s_b, s_go;
    __shared__ ResArgs s_args;
    volatile int* vc = &s_c;
    volatile int* vb = &s_b;
    volatile int* vgo = &s_go;
    for (;;) {
        __syncthreads();  // the previous pair is finished before the shared fields change
        if (threadIdx.x == 0) {
            const int w = (int)atomicAdd(a.next, 1u);
            int c = 0, b = w;
            while (c < a.n_classes - 1 && b >= a.cls[c].count) {
                b -= a.cls[c].count;
                ++c;
            }
            *vc = c;
            *vb = b;
            *vgo = w >= a.total ? 0 : (a.cls[c].ctl[b].error ? 2 : 1);
        }
        __syncthreads();
        const int go = *vgo;
        if (go == 0) return;
        if (go == 2) continue;
        const CascadeClass* K = a.cls + *vc;
        const int b = *vb;
        for (int l = 0; l < K->split; ++l) {
            const CascadeLevel& v = K->lv[l];
            cascade_init(K, l, b, 0, v.nx * v.ny);
            if (threadIdx.x == 0) cascade_args(s_args, a, K, l);
            __syncthreads();  // the level's state is in global memory for the level solve to load
            res4_level<NORM, false>(s_args, b, 1, 0, smraw);
            __syncthreads();  // the level's final state is stored before the next level reads it
        }
    }
}

static size_t cascade_coarse_smem() { return resident_smem(CASCADE_COARSE_NODES); }

static const void* cascade_coarse_fn(int norm)
{
    return norm == W1_NORM_L1 ? (const void*)k_cascade_coarse<W1_NORM_L1>
           : norm == W1_NORM_L2 ? (const void*)k_cascade_coarse<W1_NORM_L2>
                                : (const void*)k_cascade_coarse<W1_NORM_LINF>;
}

int cascade_coarse_ctas(int norm)
{
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, cascade_coarse_fn(norm), CASCADE_COARSE_THREADS,
                                                      cascade_coarse_smem()) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return sms * per;
}

cudaError_t launch_cascade_coarse(int norm, const CascadeArgs& a, int ctas, cudaStream_t s)
{
    if (ctas < 1 || a.total < 1) return cudaErrorInvalidValue;
    const int grid = ctas < a.total ? ctas : a.total;
    void* args[1] = {(void*)&a};
    return cudaLaunchKernel(cascade_coarse_fn(norm), dim3(grid), dim3(CASCADE_COARSE_THREADS), args,
                            cascade_coarse_smem(), s);
}

template <int NORM>
static cudaError_t cascade_attr()
{
    cudaError_t e = cudaFuncSetAttribute(k_cascade<NORM, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)cascade_smem(false));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_cascade<NORM, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)cascade_smem(true));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_cascade_cl<NORM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cascade_smem(true));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_cascade_coarse<NORM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)cascade_coarse_smem());
}

static const void* cascade_fn(int norm, bool wide)
{
    if (wide)
        return norm == W1_NORM_L1 ? (const void*)k_cascade<W1_NORM_L1, true>
               : norm == W1_NORM_L2 ? (const void*)k_cascade<W1_NORM_L2, true>
                                    : (const void*)k_cascade<W1_NORM_LINF, true>;
    return norm == W1_NORM_L1 ? (const void*)k_cascade<W1_NORM_L1, false>
           : norm == W1_NORM_L2 ? (const void*)k_cascade<W1_NORM_L2, false>
                                : (const void*)k_cascade<W1_NORM_LINF, false>;
}

int cascade_ctas(int norm, bool wide)
{
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, cascade_fn(norm, wide), RES_THREADS, cascade_smem(wide)) !=
            cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return sms * per;
}

cudaError_t launch_cascade(int norm, bool wide, const CascadeArgs& a, int ctas, cudaStream_t s)
{
    if (ctas < 1 || a.total < 1) return cudaErrorInvalidValue;
    const int grid = ctas < a.total ? ctas : a.total;
    void* args[1] = {(void*)&a};
    return cudaLaunchKernel(cascade_fn(norm, wide), dim3(grid), dim3(RES_THREADS), args, cascade_smem(wide), s);
}

template <int NORM, int NPT, bool CL>
static cudaError_t res_attr()
{
    cudaError_t e = cudaFuncSetAttribute(k_resident<NORM, NPT, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)resident_smem(RES_MAX_NODES));
    if (e != cudaSuccess) return e;
    if (CL) return cudaFuncSetAttribute(k_resident<NORM, NPT, CL>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return cudaSuccess;
}

template <int NORM>
static cudaError_t res_attr_norm()
{
    cudaError_t e;
    if ((e = res_attr<NORM, 1, false>()) != cudaSuccess) return e;
    if ((e = res_attr<NORM, 2, false>()) != cudaSuccess) return e;
    if ((e = res_attr<NORM, 8, false>()) != cudaSuccess) return e;
    if ((e = res_attr<NORM, 1, true>()) != cudaSuccess) return e;
    if ((e = res_attr<NORM, 2, true>()) != cudaSuccess) return e;
    return res_attr<NORM, 4, true>();
}

template <int NORM, bool CL>
static cudaError_t res4_attr()
{
    cudaError_t e = cudaFuncSetAttribute(k_resident4<NORM, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)resident_smem(RES_MAX_NODES));
    if (e != cudaSuccess) return e;
    if (CL) return cudaFuncSetAttribute(k_resident4<NORM, CL>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return cudaSuccess;
}

template <int NORM>
static cudaError_t resw_attr()
{
    cudaError_t e = cudaFuncSetAttribute(k_resident_wide<NORM, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)resident_wide_smem(RESW_MAX_NODES));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_resident_wide<NORM, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)resident_wide_smem(RESW_MAX_NODES));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_resident_wide<NORM, true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

cudaError_t resident_prepare(int)
{
    cudaError_t e = tblock_prepare();
    if (e != cudaSuccess) return e;
    e = res_attr_norm<W1_NORM_L1>();
    if (e != cudaSuccess) return e;
    if ((e = res_attr_norm<W1_NORM_L2>()) != cudaSuccess) return e;
    if ((e = res_attr_norm<W1_NORM_LINF>()) != cudaSuccess) return e;
    if ((e = res4_attr<W1_NORM_L1, false>()) != cudaSuccess) return e;
    if ((e = res4_attr<W1_NORM_L1, true>()) != cudaSuccess) return e;
    if ((e = res4_attr<W1_NORM_L2, false>()) != cudaSuccess) return e;
    if ((e = res4_attr<W1_NORM_L2, true>()) != cudaSuccess) return e;
    if ((e = res4_attr<W1_NORM_LINF, false>()) != cudaSuccess) return e;
    if ((e = res4_attr<W1_NORM_LINF, true>()) != cudaSuccess) return e;
    if ((e = resw_attr<W1_NORM_L1>()) != cudaSuccess) return e;
    if ((e = resw_attr<W1_NORM_L2>()) != cudaSuccess) return e;
    if ((e = resw_attr<W1_NORM_LINF>()) != cudaSuccess) return e;
    if ((e = cascade_attr<W1_NORM_L1>()) != cudaSuccess) return e;
    if ((e = cascade_attr<W1_NORM_L2>()) != cudaSuccess) return e;
    return cascade_attr<W1_NORM_LINF>();
}

template <int NORM>
static const void* res_fn(int npt, bool cl)
{
    if (cl) {
        if (npt <= 1) return (const void*)k_resident<NORM, 1, true>;
        if (npt <= 2) return (const void*)k_resident<NORM, 2, true>;
        return (const void*)k_resident<NORM, 4, true>;
    }
    if (npt <= 1) return (const void*)k_resident<NORM, 1, false>;
    if (npt <= 2) return (const void*)k_resident<NORM, 2, false>;
    return (const void*)k_resident<NORM, 8, false>;
}

static void resident_config(int norm, int cluster, int nx, int ny, int pairs, cudaLaunchConfig_t& cfg,
                            cudaLaunchAttribute* attr, const void** fn)
{
    const int band = (ny / cluster) * nx;
    if (band > RES_MAX_NODES) {
        // wide band: four runs of four nodes per thread
        cfg = cudaLaunchConfig_t{};
        cfg.gridDim = dim3(cluster * pairs, 1, 1);
        cfg.blockDim = dim3(RES_THREADS, 1, 1);
        cfg.dynamicSmemBytes = resident_wide_smem(band);
        cfg.numAttrs = 0;
        const bool cl = cluster > 1;
        if (cl) {
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = cluster;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
        }
        if (norm == W1_NORM_L1)
            *fn = cl ? (const void*)k_resident_wide<W1_NORM_L1, true> : (const void*)k_resident_wide<W1_NORM_L1, false>;
        else if (norm == W1_NORM_L2)
            *fn = cl ? (const void*)k_resident_wide<W1_NORM_L2, true> : (const void*)k_resident_wide<W1_NORM_L2, false>;
        else
            *fn = cl ? (const void*)k_resident_wide<W1_NORM_LINF, true>
                     : (const void*)k_resident_wide<W1_NORM_LINF, false>;
        return;
    }
    if (nx % 4 == 0 && band / 4 <= RES_THREADS) {
        // four consecutive nodes of a row per thread
        const int threads = ((band / 4 + 31) / 32) * 32;
        cfg = cudaLaunchConfig_t{};
        cfg.gridDim = dim3(cluster * pairs, 1, 1);
        cfg.blockDim = dim3(threads, 1, 1);
        cfg.dynamicSmemBytes = resident_smem(band);
        cfg.numAttrs = 0;
        if (cluster > 1) {
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = cluster;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
        }
        if (norm == W1_NORM_L1)
            *fn = cluster > 1 ? (const void*)k_resident4<W1_NORM_L1, true> : (const void*)k_resident4<W1_NORM_L1, false>;
        else if (norm == W1_NORM_L2)
            *fn = cluster > 1 ? (const void*)k_resident4<W1_NORM_L2, true> : (const void*)k_resident4<W1_NORM_L2, false>;
        else
            *fn = cluster > 1 ? (const void*)k_resident4<W1_NORM_LINF, true>
                              : (const void*)k_resident4<W1_NORM_LINF, false>;
        return;
    }
    // up to 1024 nodes: one per thread; up to 2048: two per thread; beyond:
    // 512 threads x 8 for a single CTA, 1024 x 4 in a cluster (fewer registers
    // next to the distributed-shared-memory addressing)
    int threads, npt;
    if (band <= RES_THREADS) {
        threads = ((band + 31) / 32) * 32;
        npt = 1;
    } else if (band <= 2 * RES_THREADS) {
        threads = RES_THREADS;
        npt = 2;
    } else if (cluster > 1) {
        threads = RES_THREADS;
        npt = 4;
    } else {
        threads = RES_THREADS / 2;
        npt = 8;
    }
    cfg = cudaLaunchConfig_t{};
    cfg.gridDim = dim3(cluster * pairs, 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = resident_smem(band);
    cfg.numAttrs = 0;
    if (cluster > 1) {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cluster;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    *fn = norm == W1_NORM_L1   ? res_fn<W1_NORM_L1>(npt, cluster > 1)
          : norm == W1_NORM_L2 ? res_fn<W1_NORM_L2>(npt, cluster > 1)
                               : res_fn<W1_NORM_LINF>(npt, cluster > 1);
}

int resident_cluster_ok(int norm, int cluster, int nx, int ny)
{
    if (!resident_fits(nx, ny, cluster)) return 0;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    const void* fn = nullptr;
    resident_config(norm, cluster, nx, ny, 1, cfg, attr, &fn);
    int n = 0;
    if (cluster == 1) {
        // single CTAs: resident blocks per SM times SMs
        int dev = 0, sms = 0, per = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, (int)(cfg.blockDim.x), cfg.dynamicSmemBytes) !=
                cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return sms * per;
    }
    if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

cudaError_t launch_resident(int norm, int cluster, const ResArgs& a, cudaStream_t s)
{
    if (!resident_fits(a.it.nx, a.it.ny, cluster)) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    const void* fn = nullptr;
    resident_config(norm, cluster, a.it.nx, a.it.ny, a.pairs, cfg, attr, &fn);
    cfg.stream = s;
    void* args[1] = {(void*)&a};
    return cudaLaunchKernelExC(&cfg, fn, args);
}

// ---------------------------------------------------------------------------
// Final statistics: W1 = f(m), dual bound, residual, certified bracket
// ---------------------------------------------------------------------------

static constexpr int FIN_THREADS = 256;

// At most FIN_BLOCKS_PER_PAIR blocks per pair, from the grid alone (same reason
// as the prep blocks); each leaves FIN_PART_PER_BLOCK doubles (w1_internal.h).
static int final_blocks_per_pair(int) { return FIN_BLOCKS_PER_PAIR; }

size_t final_part_doubles(int pairs) { return (size_t)final_blocks_per_pair(pairs) * pairs * FIN_PART_PER_BLOCK; }

// Grids whose sides are multiples of FIN_TILE do the first five levels of the
// route bound inside k_final_a, one FIN_TILE x FIN_TILE tile per block step
// ((FIN_TILE / 2)^2 = FIN_THREADS cells of 2 x 2 nodes, one per thread).
static constexpr int FIN_TILE = 32;
static_assert((FIN_TILE / 2) * (FIN_TILE / 2) == FIN_THREADS, "one 2x2 cell per thread");

// Nodes per side that k_final_a pools before k_final_b continues the tree.
__host__ __device__ static inline int final_pool(int nx, int ny)
{
    if (nx % FIN_TILE == 0 && ny % FIN_TILE == 0) return FIN_TILE;
    return ((nx & 1) == 0 && (ny & 1) == 0) ? 2 : 1;
}

// Per node (FP64 from the FP32 state; e = rho - div m the constraint residual):
//   ||m(x)||_p, phi rho, |e|, |rho|, phi e, and ||grad phi(x)||_q.
// Each sum is compensated and left unscaled; h^2 is applied once at the end.
// The signed sums (phi rho, phi e) add every node's term to their compensated
// sum; the non-negative ones (||m||_p, |e|, |rho|, route costs) add a 2 x 2
// cell's terms in plain FP64 first (relative error at most 3 units of
// roundoff, which no cancellation can amplify) and that to the compensated
// sum.  Every term except the p = 2 norm and e is exact in FP64 (products and
// sums of two FP32 values); 1/h multiplies instead of dividing by h (one
// rounding more where h is not a power of two).  For p = 2 the running maximum
// of ||grad phi||_2 is kept squared, with one square root per block (the
// square root is monotone and correctly rounded, so the maximum is the same).
// When nx and ny are both even each thread takes 2 x 2 cells and also does the
// first level of the route bound (see k_final_b): the cost of sending each
// node's residual mass to its cell's first node; with both sides multiples of
// FIN_TILE the block carries the tree on to one node per tile.  The masses
// left (per cell or per tile) go to q, compactly, for k_final_b.
template <int NORM>
__global__ void __launch_bounds__(FIN_THREADS) k_final_a(const float* __restrict__ m1, const float* __restrict__ m2,
                                                         const float* __restrict__ phi, const float* __restrict__ rho,
                                                         int nx, int ny, double h, double* __restrict__ q,
                                                         double* part, const Ctl* ctls)
{
    __shared__ double sh[2 * 6 * FIN_THREADS];
    __shared__ double tq[2][FIN_THREADS];
    const int pair = blockIdx.y;
    if (ctls && ctls[pair].error == 2) return;
    const long long n = (long long)nx * ny;
    const size_t off = (size_t)pair * n;
    m1 += off;
    m2 += off;
    phi += off;
    rho += off;
    q += 2 * off;
    CSum v[6];  // sum ||m||_p, sum phi rho, sum |e|, sum |rho|, sum phi e, route cost
    double gm = 0.0;  // max ||grad phi||_q (squared for p = 2)
    const double h2 = h * h, inv_h = 1.0 / h;
    // the node's terms (non-negative ones into acc); returns its residual mass e h^2
    auto node = [&](int i, int j, double (&acc)[3]) -> double {
        const long long k = (long long)j * nx + i;
        const double a1 = (i < nx - 1) ? (double)m1[k] : 0.0;
        const double a2 = (j < ny - 1) ? (double)m2[k] : 0.0;
        acc[0] += NORM == W1_NORM_L1     ? __dadd_rn(fabs(a1), fabs(a2))
                  : NORM == W1_NORM_LINF ? fmax(fabs(a1), fabs(a2))
                                         : sqrt(__dadd_rn(__dmul_rn(a1, a1), __dmul_rn(a2, a2)));
        const double p = phi[k], r = rho[k];
        v[1].add(__dmul_rn(p, r));
        double d = __dadd_rn(a1, a2);
        if (i > 0) d = __dsub_rn(d, (double)m1[k - 1]);
        if (j > 0) d = __dsub_rn(d, (double)m2[k - nx]);
        const double e = __dsub_rn(r, __dmul_rn(d, inv_h));
        acc[1] += fabs(e);
        acc[2] += fabs(r);
        v[4].add(__dmul_rn(p, e));
        const double g1 = (i < nx - 1) ? __dmul_rn((double)phi[k + 1] - p, inv_h) : 0.0;
        const double g2 = (j < ny - 1) ? __dmul_rn((double)phi[k + nx] - p, inv_h) : 0.0;
        const double gq = (NORM == W1_NORM_L1) ? fmax(fabs(g1), fabs(g2))
                          : (NORM == W1_NORM_LINF ? fabs(g1) + fabs(g2) : g1 * g1 + g2 * g2);
        gm = fmax(gm, gq);
        return e * h2;
    };
    auto flush = [&](const double (&acc)[3]) {
        v[0].add(acc[0]);
        v[2].add(acc[1]);
        v[3].add(acc[2]);
    };
    // a 2 x 2 cell with first node (i, j): its terms and the first route
    // level (offsets (1,0) and (0,1) cost one edge hl, (1,1) two); returns the
    // cell's mass.  The same step, on masses, serves the coarser levels.
    auto pool4 = [&](double a00, double a10, double a01, double a11, double hl) -> double {
        v[5].add(__dmul_rn(__dadd_rn(__dadd_rn(fabs(a10), fabs(a01)), __dmul_rn(2.0, fabs(a11))), hl));
        return ((a00 + a10) + a01) + a11;
    };
    auto cell = [&](int i, int j) -> double {
        double acc[3] = {0.0, 0.0, 0.0};
        const double q00 = node(i, j, acc), q10 = node(i + 1, j, acc);
        const double q01 = node(i, j + 1, acc), q11 = node(i + 1, j + 1, acc);
        flush(acc);
        return pool4(q00, q10, q01, q11, h);
    };
    const long long stride = (long long)gridDim.x * blockDim.x;
    const int pool = final_pool(nx, ny);
    if (pool == FIN_TILE) {
        const int tx = nx / FIN_TILE, ntile = tx * (ny / FIN_TILE);
        const int half0 = FIN_TILE / 2, ci = threadIdx.x % half0, cj = threadIdx.x / half0;
        for (int t = blockIdx.x; t < ntile; t += gridDim.x) {  // uniform over the block
            const int TJ = t / tx, TI = t - TJ * tx;
            tq[0][threadIdx.x] = cell(TI * FIN_TILE + 2 * ci, TJ * FIN_TILE + 2 * cj);
            // the tile's cells down to one node: side 16 -> 8 -> 4 -> 2 -> 1 (ping-pong
            // buffers; the barrier before each level orders it after the last one)
            int side = half0, src = 0;
            double hl = 2.0 * h;
            while (side > 1) {
                __syncthreads();
                const int half = side / 2;
                if ((int)threadIdx.x < half * half) {
                    const int J = threadIdx.x / half, I = threadIdx.x - J * half;
                    const double* sq = tq[src] + 2 * J * side + 2 * I;
                    tq[src ^ 1][threadIdx.x] = pool4(sq[0], sq[1], sq[side], sq[side + 1], hl);
                }
                src ^= 1;
                side = half;
                hl *= 2.0;
            }
            // thread 0 wrote the last level itself; the next tile's cells overwrite
            // only entries no thread reads any more
            if (threadIdx.x == 0) q[t] = tq[src][0];
        }
    } else if (pool == 2) {
        const int ncx = nx / 2;
        const long long nc = n / 4;
        for (long long kb = blockIdx.x * (long long)blockDim.x + threadIdx.x; kb < nc; kb += stride) {
            const int J = (int)(kb / ncx), I = (int)(kb - (long long)J * ncx);
            q[kb] = cell(2 * I, 2 * J);
        }
    } else {
        for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += stride) {
            const int j = (int)(k / nx), i = (int)(k - (long long)j * nx);
            double acc[3] = {0.0, 0.0, 0.0};
            q[k] = node(i, j, acc);
            flush(acc);
        }
    }
    block_csum_sh<6>(v, sh);
    gm = warp_max(gm);
    __shared__ double shm[32];
    if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = gm;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) gm = fmax(gm, shm[w]);
        double* pp = part + ((size_t)pair * gridDim.x + blockIdx.x) * FIN_PART_PER_BLOCK;
        for (int c = 0; c < 6; ++c) {
            pp[2 * c] = v[c].s;
            pp[2 * c + 1] = v[c].c;
        }
        pp[12] = NORM == W1_NORM_L2 ? sqrt(gm) : gm;
    }
}

// One block per pair: sums the partials (compensated), then routes the
// residual masses q along the dyadic tree (each 2x2 block sends its masses to
// its first node; offsets (1,0), (0,1) cost one edge of the current spacing,
// (1,1) two), finishing with a diameter bound on the last grid.  This is an
// explicit flux carrying rho - div m, hence f + route >= W1 of the discrete
// problem.  The saddle value is the Lagrangian of eq. minmax_cp at the state,
// L(m, phi) = f(m) + <phi, div m - rho>_h = h^2 (sum ||m||_p - sum phi e).
__global__ void __launch_bounds__(FIN_THREADS) k_final_b(int nx, int ny, double h, double* q, const double* part,
                                                         int nparts, Ctl* ctls)
{
    const int pair = blockIdx.x;
    Ctl* ctl = ctls + pair;
    if (ctl->error == 2) return;
    const size_t n = (size_t)nx * ny;
    double* src = q + 2 * n * pair;
    double* dst = src + n;
    part += (size_t)pair * nparts * FIN_PART_PER_BLOCK;
    __shared__ double sh[2 * 6 * FIN_THREADS];
    CSum v[6];
    double gm = 0.0;
    for (int b = threadIdx.x; b < nparts; b += blockDim.x) {
        for (int c = 0; c < 6; ++c) {
            CSum x;
            x.s = part[b * FIN_PART_PER_BLOCK + 2 * c];
            x.c = part[b * FIN_PART_PER_BLOCK + 2 * c + 1];
            v[c].add(x);
        }
        gm = fmax(gm, part[b * FIN_PART_PER_BLOCK + 12]);
    }
    block_csum_sh<6>(v, sh);
    __shared__ double tot[5], sad;
    __shared__ CSum cost0;
    if (threadIdx.x == 0) {
        for (int c = 0; c < 5; ++c) tot[c] = v[c].value();
        CSum lag = v[0], pe;
        pe.s = -v[4].s;
        pe.c = -v[4].c;
        lag.add(pe);
        sad = lag.value();
        cost0 = v[5];
    }
    gm = warp_max(gm);
    __shared__ double shm[32];
    if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = gm;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) gm = fmax(gm, shm[w]);

    // k_final_a did the first levels of the tree: one (both sides even) or
    // five (both sides multiples of FIN_TILE)
    const int pool = final_pool(nx, ny);
    int cx = nx / pool, cy = ny / pool;
    double hx = pool * h, hy = pool * h;
    CSum cost;
    for (;;) {
        const int px = (cx > 1 && (cx & 1) == 0), py = (cy > 1 && (cy & 1) == 0);
        const int stopx = (cx > 1 && (cx & 1)), stopy = (cy > 1 && (cy & 1));
        if (stopx || stopy || (!px && !py)) break;
        const int bx = px ? 2 : 1, by = py ? 2 : 1;
        const int ncx = cx / bx, ncy = cy / by;
        const int nc = ncx * ncy;  // grids of up to 2^31 nodes
        const double w[2][2] = {{0.0, hx}, {hy, hx + hy}};  // distance to the block's corner
        for (int k = threadIdx.x; k < nc; k += blockDim.x) {
            const int J = k / ncx, I = k - J * ncx;
            double total = 0.0, cs = 0.0;  // the block's costs are non-negative: one compensated add
            for (int b = 0; b < by; ++b)
                for (int a = 0; a < bx; ++a) {
                    const double qa = src[(size_t)(by * J + b) * cx + (bx * I + a)];
                    if (a | b) cs += __dmul_rn(fabs(qa), w[b][a]);
                    total += qa;
                }
            cost.add(cs);
            dst[k] = total;
        }
        __syncthreads();
        double* t = src;
        src = dst;
        dst = t;
        cx = ncx;
        cy = ncy;
        if (px) hx *= 2.0;
        if (py) hy *= 2.0;
    }
    CSum ws[3];
    ws[0] = cost;
    if (threadIdx.x == 0) ws[0].add(cost0);
    for (int k = threadIdx.x; k < cx * cy; k += blockDim.x) {
        const double x = src[k];
        if (x > 0) ws[1].add(x);
        else ws[2].add(-x);
    }
    block_csum_sh<3>(ws, sh);
    if (threadIdx.x == 0) {
        const double h2 = h * h;
        const double diam = (cx - 1) * hx + (cy - 1) * hy;
        const double route = ws[0].value() + diam * fmax(ws[1].value(), ws[2].value());
        ctl->f = tot[0] * h2;
        ctl->dual = -tot[1] * h2;
        ctl->res_l1 = tot[2] * h2;
        ctl->rho_l1 = tot[3] * h2;
        ctl->saddle = sad * h2;
        ctl->gmax = gm;
        ctl->route = route;
        ctl->lb = ctl->dual / fmax(1.0, gm);
        ctl->ub = ctl->f + route;
    }
}

cudaError_t launch_final(int norm, const float* m1, const float* m2, const float* phi, const float* rho, int nx,
                         int ny, double h, double* q, double* part, Ctl* ctl, int pairs, cudaStream_t s)
{
    // one block per 32 x 32 tile, or per 1024 cells (nodes, or 2 x 2 blocks of
    // nodes), at most FIN_BLOCKS_PER_PAIR: each block ends with a block-wide FP64 sum
    const int pool = final_pool(nx, ny);
    const long long units = pool == FIN_TILE ? (long long)(nx / FIN_TILE) * (ny / FIN_TILE)
                                             : ((long long)nx * ny / (pool * pool) + 1023) / 1024;
    const int bpp = (int)(units < 1 ? 1 : units > FIN_BLOCKS_PER_PAIR ? FIN_BLOCKS_PER_PAIR : units);
    dim3 g(bpp, pairs);
    if (norm == W1_NORM_L1)
        k_final_a<W1_NORM_L1><<<g, FIN_THREADS, 0, s>>>(m1, m2, phi, rho, nx, ny, h, q, part, ctl);
    else if (norm == W1_NORM_L2)
        k_final_a<W1_NORM_L2><<<g, FIN_THREADS, 0, s>>>(m1, m2, phi, rho, nx, ny, h, q, part, ctl);
    else
        k_final_a<W1_NORM_LINF><<<g, FIN_THREADS, 0, s>>>(m1, m2, phi, rho, nx, ny, h, q, part, ctl);
    k_final_b<<<pairs, FIN_THREADS, 0, s>>>(nx, ny, h, q, part, bpp, ctl);
    return cudaGetLastError();
}

}  // namespace w1
