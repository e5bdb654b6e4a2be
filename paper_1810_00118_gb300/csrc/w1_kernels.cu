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
//   * resident: a whole level lives in shared memory and registers of one CTA
//     or of a thread-block cluster (bands of rows, halo rows read through
//     distributed shared memory); all iterations and stop tests of the level run
//     inside one launch, two cluster barriers per step.
//   * streaming: one launch per step over global memory (ping-pong buffers);
//     each warp covers 32 columns and marches up a strip of rows, carrying the
//     row below in registers and exchanging the left/right neighbours by warp
//     shuffles, so every value is read once per step (28 B/node/step).
// Reductions are FP64 with a fixed summation order (deterministic).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "w1_internal.h"

namespace cg = cooperative_groups;

namespace w1 {

static constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------------------
// Proximal maps (the argmin of the first line of eq. primaldual)
// ---------------------------------------------------------------------------

__device__ __forceinline__ float soft(float v, float mu)
{
    float a = fabsf(v) - mu;
    return a > 0.f ? copysignf(a, v) : 0.f;
}

template <int NORM>
__device__ __forceinline__ void prox(float v1, float v2, float mu, float& o1, float& o2)
{
    if (NORM == W1_NORM_L1) {
        o1 = soft(v1, mu);
        o2 = soft(v2, mu);
    } else {
        float len = sqrtf(v1 * v1 + v2 * v2);
        float s = (len > mu) ? 1.f - mu / len : 0.f;
        o1 = v1 * s;
        o2 = v2 * s;
    }
}

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Warp / block reductions in a fixed order.
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(FULL, v, o));
    return v;
}

// Sums N values over the block; result valid in thread 0.  sh: 32*N doubles.
template <int N>
__device__ void block_sum(double (&v)[N], double* sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int c = 0; c < N; ++c) v[c] = warp_sum(v[c]);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < N; ++c) sh[warp * N + c] = v[c];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int c = 0; c < N; ++c) {
            double x = (lane < nw) ? sh[lane * N + c] : 0.0;
            v[c] = warp_sum(x);
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Prep: rho = rho0 - rho1 (Sec. 2.2), mass check, exact zero mean
// ---------------------------------------------------------------------------

static constexpr int PREP_BLOCKS = 304, PREP_THREADS = 256;

__global__ void __launch_bounds__(PREP_THREADS) k_prep_reduce(const float* __restrict__ r0,
                                                              const float* __restrict__ r1, long long n, double h,
                                                              Ctl* ctl, double* part)
{
    __shared__ double sh[32 * 4];
    __shared__ bool last;
    double v[4] = {0.0, 0.0, 0.0, 0.0};  // sum r0, sum r1, sum (r0 - r1), non-finite count
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        float a = r0[k], b = r1[k];
        if (!isfinite(a) || !isfinite(b)) v[3] += 1.0;
        v[0] += a;
        v[1] += b;
        v[2] += (double)a - (double)b;
    }
    block_sum<4>(v, sh);
    if (threadIdx.x == 0) {
        for (int c = 0; c < 4; ++c) part[blockIdx.x * 4 + c] = v[c];
        __threadfence();
        last = (atomicAdd(&ctl->counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double t[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
        for (int c = 0; c < 4; ++c) t[c] += ((volatile double*)part)[b * 4 + c];
    block_sum<4>(t, sh);
    if (threadIdx.x == 0) {
        double M0 = t[0] * h * h, M1 = t[1] * h * h;
        ctl->mass0 = M0;
        ctl->mass1 = M1;
        ctl->mean = t[2] / (double)n;
        int bad = (t[3] > 0.0) || !(fabs(M0 - M1) <= 1e-6 * fmax(fabs(M0), fabs(M1)));
        ctl->error = bad;
        ctl->timeout = 0;
        ctl->counter = 0;
    }
}

__global__ void k_prep_apply(const float* __restrict__ r0, const float* __restrict__ r1, long long n,
                             const Ctl* __restrict__ ctl, float* __restrict__ rho)
{
    const double mean = ctl->mean;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        rho[k] = (float)(((double)r0[k] - (double)r1[k]) - mean);
}

cudaError_t launch_prep(const float* r0, const float* r1, long long n, double h, Ctl* ctl, double* part,
                        float* rho, cudaStream_t s)
{
    k_prep_reduce<<<PREP_BLOCKS, PREP_THREADS, 0, s>>>(r0, r1, n, h, ctl, part);
    k_prep_apply<<<PREP_BLOCKS * 2, 256, 0, s>>>(r0, r1, n, ctl, rho);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Restriction (2x2 block mean) and Interpolate (Sec. 3.3, pixel-grid reading)
// ---------------------------------------------------------------------------

__global__ void k_restrict(const float* __restrict__ f, int nx, int ny, float* __restrict__ c)
{
    const int ncx = nx / 2, ncy = ny / 2;
    const int I = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y * blockDim.y + threadIdx.y;
    if (I >= ncx || J >= ncy) return;
    const float* r0 = f + (size_t)(2 * J) * nx + 2 * I;
    const float* r1 = r0 + nx;
    c[(size_t)J * ncx + I] = 0.25f * ((r0[0] + r0[1]) + (r1[0] + r1[1]));
}

cudaError_t launch_restrict(const float* fine, int nx, int ny, float* coarse, cudaStream_t s)
{
    dim3 b(32, 8), g((nx / 2 + 31) / 32, (ny / 2 + 7) / 8);
    k_restrict<<<g, b, 0, s>>>(fine, nx, ny, coarse);
    return cudaGetLastError();
}

// phi: bilinear on cell centres (3/4 own coarse cell, 1/4 the neighbour on the
// fine node's side, clamped); m1: odd fine x-edges copy the coarse x-edge they
// lie on, even ones average the coarse x-edges around their coarse cell, rows
// copy; m2 likewise with the axes exchanged.
__global__ void k_prolong(int ncx, int ncy, const float* __restrict__ m1c, const float* __restrict__ m2c,
                          const float* __restrict__ phic, float* __restrict__ m1f, float* __restrict__ m2f,
                          float* __restrict__ phif)
{
    const int nx = 2 * ncx, ny = 2 * ncy;
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= nx || j >= ny) return;
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

cudaError_t launch_prolong(int ncx, int ncy, const float* m1c, const float* m2c, const float* phic, float* m1f,
                           float* m2f, float* phif, cudaStream_t s)
{
    dim3 b(32, 8), g((2 * ncx + 31) / 32, (2 * ncy + 7) / 8);
    k_prolong<<<g, b, 0, s>>>(ncx, ncy, m1c, m2c, phic, m1f, m2f, phif);
    return cudaGetLastError();
}

__global__ void k_level_begin(Ctl* ctl, int level)
{
    ctl->iters[level] = 0;
    ctl->fpr[level] = 0.0;
    ctl->conv[level] = 0;
    ctl->t_start[level] = globaltimer();
}

cudaError_t launch_level_begin(Ctl* ctl, int level, cudaStream_t s)
{
    k_level_begin<<<1, 1, 0, s>>>(ctl, level);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Streaming step (one step of eq. primaldual over global memory)
// ---------------------------------------------------------------------------

static constexpr int STEP_THREADS = 256;  // 8 warps stacked in y

int stream_rows_auto(int nx, int ny)
{
    // enough blocks for ~4 waves of 152 SMs, marching at most 16 rows per thread
    long long colblocks = (nx + 31) / 32;
    long long r = (long long)ny * colblocks / (8LL * 152 * 4);
    if (r < 2) r = 2;
    if (r > 16) r = 16;
    return (int)r;
}

dim3 stream_grid(int nx, int ny, int rows)
{
    return dim3((nx + 31) / 32, (ny + 8 * rows - 1) / (8 * rows), 1);
}

size_t step_part_doubles(int nx, int ny, int rows)
{
    dim3 g = stream_grid(nx, ny, rows);
    return (size_t)g.x * g.y * 3;
}

template <int NORM, bool CHECK>
__global__ void __launch_bounds__(STEP_THREADS) k_step(StepArgs a)
{
    const IterArgs& P = a.it;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nx = P.nx, ny = P.ny;
    const int i = blockIdx.x * 32 + lane;
    const int j0 = (blockIdx.y * (STEP_THREADS / 32) + warp) * a.rows;
    const bool act = i < nx;
    const float mu = P.mu, tau = P.tau, ih = P.ih;
    double sa = 0.0, sb = 0.0, sc = 0.0;
    const bool err = P.ctl != nullptr && P.ctl->error != 0;
    if (!err && j0 < ny) {
        const int j1 = min(j0 + a.rows, ny);
        const float* __restrict__ phi = a.phi;
        const float* __restrict__ m1 = a.m1;
        const float* __restrict__ m2 = a.m2;
        const float* __restrict__ rho = a.rho;
        auto at = [nx](int j, int ii) { return (size_t)j * nx + ii; };
        float pc = act ? __ldg(phi + at(j0, i)) : 0.f;
        // mbar2 and dm2 of the node below the strip (row j0 - 1)
        float b2b = 0.f;
        double d2b = 0.0;
        if (j0 > 0) {
            float pb = act ? __ldg(phi + at(j0 - 1, i)) : 0.f;
            float c2 = act ? __ldg(m2 + at(j0 - 1, i)) : 0.f;
            float g2 = (pc - pb) * ih;
            float o1, o2;
            if (NORM == W1_NORM_L1) {
                o2 = soft(c2 + mu * g2, mu);
            } else {
                float pbr = __shfl_down_sync(FULL, pb, 1);
                if (lane == 31 && i + 1 < nx) pbr = __ldg(phi + at(j0 - 1, i + 1));
                float g1 = (i < nx - 1) ? (pbr - pb) * ih : 0.f;
                float c1 = act ? __ldg(m1 + at(j0 - 1, i)) : 0.f;
                prox<NORM>(c1 + mu * g1, c2 + mu * g2, mu, o1, o2);
            }
            b2b = 2.f * o2 - c2;
            d2b = (double)o2 - (double)c2;
        }
        for (int j = j0; j < j1; ++j) {
            const float pu = (act && j + 1 < ny) ? __ldg(phi + at(j + 1, i)) : 0.f;
            float pr = __shfl_down_sync(FULL, pc, 1);
            if (lane == 31 && i + 1 < nx) pr = __ldg(phi + at(j, i + 1));
            const float a1 = act ? __ldg(m1 + at(j, i)) : 0.f;
            const float a2 = act ? __ldg(m2 + at(j, i)) : 0.f;
            const float r = act ? __ldg(rho + at(j, i)) : 0.f;
            const float g1 = (i < nx - 1) ? (pr - pc) * ih : 0.f;
            const float g2 = (j < ny - 1) ? (pu - pc) * ih : 0.f;
            float n1, n2;
            prox<NORM>(a1 + mu * g1, a2 + mu * g2, mu, n1, n2);
            if (i >= nx - 1) n1 = 0.f;
            if (j == ny - 1) n2 = 0.f;
            const float b1 = 2.f * n1 - a1, b2 = 2.f * n2 - a2;
            float b1l = __shfl_up_sync(FULL, b1, 1);
            double d1l = 0.0;
            if (CHECK) d1l = __shfl_up_sync(FULL, (double)n1 - (double)a1, 1);
            if (lane == 0) {
                if (i > 0) {
                    // the left neighbour belongs to the previous warp: recompute its m1'
                    const float ql = __ldg(phi + at(j, i - 1));
                    const float c1 = __ldg(m1 + at(j, i - 1));
                    const float gl1 = (pc - ql) * ih;
                    float o1, o2;
                    if (NORM == W1_NORM_L1) {
                        o1 = soft(c1 + mu * gl1, mu);
                    } else {
                        const float qlu = (j + 1 < ny) ? __ldg(phi + at(j + 1, i - 1)) : 0.f;
                        const float c2 = __ldg(m2 + at(j, i - 1));
                        const float gl2 = (j < ny - 1) ? (qlu - ql) * ih : 0.f;
                        prox<NORM>(c1 + mu * gl1, c2 + mu * gl2, mu, o1, o2);
                    }
                    b1l = 2.f * o1 - c1;
                    d1l = (double)o1 - (double)c1;
                } else {
                    b1l = 0.f;
                    d1l = 0.0;
                }
            }
            const float dv = ((b1 - b1l) + (b2 - b2b)) * ih;
            const float pn = pc + tau * (dv - r);
            if (act) {
                a.m1o[at(j, i)] = n1;
                a.m2o[at(j, i)] = n2;
                a.phio[at(j, i)] = pn;
            }
            if (CHECK && act) {
                const double e1 = (double)n1 - (double)a1, e2 = (double)n2 - (double)a2;
                const double ep = (double)pn - (double)pc;
                const double dd = ((e1 - d1l) + (e2 - d2b)) / P.h;
                sa += e1 * e1 + e2 * e2;
                sb += ep * ep;
                sc += ep * dd;
                d2b = e2;
            }
            b2b = b2;
            pc = pu;
        }
    }
    if (!CHECK) return;

    // R^k = (|dm|^2 / mu + |dphi|^2 / tau - 2 <dphi, div dm>) h^2   (eq. pd_stop)
    __shared__ double sh[32 * 3];
    __shared__ bool last;
    double v[3] = {sa, sb, sc};
    block_sum<3>(v, sh);
    const int nblk = gridDim.x * gridDim.y;
    const int bid = blockIdx.y * gridDim.x + blockIdx.x;
    if (threadIdx.x == 0) {
        a.part[bid * 3 + 0] = v[0];
        a.part[bid * 3 + 1] = v[1];
        a.part[bid * 3 + 2] = v[2];
        __threadfence();
        last = (atomicAdd(&P.ctl->counter, 1u) == (unsigned)nblk - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double t[3] = {0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblk; b += blockDim.x)
        for (int c = 0; c < 3; ++c) t[c] += ((volatile double*)a.part)[b * 3 + c];
    block_sum<3>(t, sh);
    if (threadIdx.x == 0) {
        Ctl* ctl = P.ctl;
        const double h2 = P.h * P.h;
        const double R = (t[0] / (double)P.mu + t[1] / (double)P.tau - 2.0 * t[2]) * h2;
        ctl->counter = 0;
        if (P.fpr_out) *P.fpr_out = R;
        if (a.use_cond) {
            const long long it = ctl->iters[P.level] + P.K;
            ctl->iters[P.level] = it;
            ctl->fpr[P.level] = R;
            const int conv = R < P.tol;
            ctl->conv[P.level] = conv;
            const bool late = (globaltimer() - ctl->t_start[P.level]) > P.budget_ns;
            if (late && !conv) ctl->timeout = 1;
            const bool go = !conv && it < P.cap && !late && ctl->error == 0;
            cudaGraphSetConditional(a.cond, go ? 1u : 0u);
        }
    }
}

cudaError_t launch_step(int norm, bool check, const StepArgs& a, cudaStream_t s)
{
    dim3 g = stream_grid(a.it.nx, a.it.ny, a.rows);
    if (norm == W1_NORM_L1) {
        if (check) k_step<W1_NORM_L1, true><<<g, STEP_THREADS, 0, s>>>(a);
        else k_step<W1_NORM_L1, false><<<g, STEP_THREADS, 0, s>>>(a);
    } else {
        if (check) k_step<W1_NORM_L2, true><<<g, STEP_THREADS, 0, s>>>(a);
        else k_step<W1_NORM_L2, false><<<g, STEP_THREADS, 0, s>>>(a);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Resident level solver: Algorithm 1 to its stop test inside one launch
// ---------------------------------------------------------------------------
//
// A cluster of C CTAs holds one level; CTA r owns rows [r*ny/C, (r+1)*ny/C).
// The band lives in shared memory: rho, phi, m (m1, m2), D = div m^k and, on
// test steps, dm = m' - m.  One step:
//   phase A: m' from m and phi (own, right, up; the row above the band is read
//            from the next CTA's shared memory), m <- m' in place;  cluster barrier
//   phase B: Dn = div m' (left, below; the row below the band from the previous
//            CTA), div mbar = 2 Dn - D, phi' = phi + tau (div mbar - rho),
//            D <- Dn, phi <- phi' in place;                       cluster barrier
// Phase A only reads other nodes' phi and phase B only other nodes' m, so the
// in-place updates are safe between the barriers.
// Stop tests: each CTA's FP64 partials go to CTA 0, which decides; every CTA
// reads the decision, so all leave the loop after the same step.

static constexpr int RES_MAX_NODES = 4096;  // nodes per CTA
static constexpr int RES_THREADS = 1024;
static constexpr int RES_RED_BYTES = 1024;  // 32 warps x 3 doubles
static constexpr int RES_SLOT_BYTES = 512;  // 16 CTAs x 3 doubles + decision

int resident_max_nodes() { return RES_MAX_NODES; }

int resident_cluster_for(int nx, int ny)
{
    const int cs[5] = {1, 2, 4, 8, 16};
    if (nx > 65535) return 0;
    for (int c : cs) {
        if (ny % c != 0) continue;
        long long band = (long long)(ny / c) * nx;
        if (band <= RES_MAX_NODES) return c;
    }
    return 0;
}

static size_t resident_smem(int band)
{
    return RES_RED_BYTES + RES_SLOT_BYTES + (size_t)band * 7 * sizeof(float);
}

template <int NORM>
__global__ void __launch_bounds__(RES_THREADS, 1) k_resident(ResArgs a)
{
    cg::cluster_group cl = cg::this_cluster();
    const IterArgs& P = a.it;
    const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
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
    if (P.ctl != nullptr && P.ctl->error != 0) return;  // uniform over the cluster

    const float mu = P.mu, tau = P.tau, ih = P.ih;
    const int T = blockDim.x;
    for (int idx = threadIdx.x; idx < nb; idx += T) {
        const size_t g = (size_t)jb * nx + idx;
        s1[idx] = a.m1[g];
        s2[idx] = a.m2[g];
        ph[idx] = a.phi[g];
        rs[idx] = a.rho[g];
    }
    cl.sync();
    const float* ph_up = (rank + 1 < C) ? cl.map_shared_rank(ph, rank + 1) : nullptr;
    const float* s2_dn = (rank > 0) ? cl.map_shared_rank(s2, rank - 1) : nullptr;
    const float* e2_dn = (rank > 0) ? cl.map_shared_rank(e2s, rank - 1) : nullptr;
    double* slots0 = cl.map_shared_rank(slots, 0);
    const int last_row = (rows - 1) * nx;

    // D^0 = div m^0
    for (int idx = threadIdx.x; idx < nb; idx += T) {
        const int jl = idx / nx, i = idx - jl * nx;
        const float l1 = i > 0 ? s1[idx - 1] : 0.f;
        const float d2 = jl > 0 ? s2[idx - nx] : (rank > 0 ? s2_dn[last_row + i] : 0.f);
        Ds[idx] = ((s1[idx] - l1) + (s2[idx] - d2)) * ih;
    }
    cl.sync();

    unsigned long long t0 = 0;
    if (rank == 0 && threadIdx.x == 0) t0 = globaltimer();
    long long it = 0;
    double R = 0.0;
    int conv = 0, late = 0;
    const long long cap = P.cap;
    while (it < cap) {
        const bool check = P.fixed ? (it + 1 == cap) : ((it + 1) % P.K == 0);
        double sa = 0.0, sb = 0.0, sc = 0.0;
        // phase A: m' = prox(m + mu grad phi)
        for (int idx = threadIdx.x; idx < nb; idx += T) {
            const int jl = idx / nx, i = idx - jl * nx, j = jb + jl;
            const float pc = ph[idx];
            float g1 = 0.f, g2 = 0.f;
            if (i < nx - 1) g1 = (ph[idx + 1] - pc) * ih;
            if (j < ny - 1) g2 = ((jl < rows - 1 ? ph[idx + nx] : ph_up[i]) - pc) * ih;
            const float a1 = s1[idx], a2 = s2[idx];
            float n1, n2;
            prox<NORM>(a1 + mu * g1, a2 + mu * g2, mu, n1, n2);
            if (i == nx - 1) n1 = 0.f;
            if (j == ny - 1) n2 = 0.f;
            if (check) {
                const float d1 = n1 - a1, d2 = n2 - a2;
                e1s[idx] = d1;
                e2s[idx] = d2;
                sa += (double)d1 * d1 + (double)d2 * d2;
            }
            s1[idx] = n1;
            s2[idx] = n2;
        }
        cl.sync();
        // phase B: phi' = phi + tau (div(2m' - m) - rho)
        for (int idx = threadIdx.x; idx < nb; idx += T) {
            const int jl = idx / nx, i = idx - jl * nx;
            const float l1 = i > 0 ? s1[idx - 1] : 0.f;
            const float d2 = jl > 0 ? s2[idx - nx] : (rank > 0 ? s2_dn[last_row + i] : 0.f);
            const float Dn = ((s1[idx] - l1) + (s2[idx] - d2)) * ih;
            const float pc = ph[idx];
            const float pn = pc + tau * ((2.f * Dn - Ds[idx]) - rs[idx]);
            if (check) {
                const double el = i > 0 ? (double)e1s[idx - 1] : 0.0;
                const double eb = jl > 0 ? (double)e2s[idx - nx] : (rank > 0 ? (double)e2_dn[last_row + i] : 0.0);
                const double dd = (((double)e1s[idx] - el) + ((double)e2s[idx] - eb)) / P.h;
                const double ep = (double)pn - (double)pc;
                sb += ep * ep;
                sc += ep * dd;
            }
            Ds[idx] = Dn;
            ph[idx] = pn;
        }
        cl.sync();
        ++it;
        if (check) {
            double v[3] = {sa, sb, sc};
            block_sum<3>(v, red);
            if (threadIdx.x == 0) {
                slots0[rank * 3 + 0] = v[0];
                slots0[rank * 3 + 1] = v[1];
                slots0[rank * 3 + 2] = v[2];
            }
            cl.sync();
            if (rank == 0 && threadIdx.x == 0) {
                double t[3] = {0.0, 0.0, 0.0};
                for (int r = 0; r < C; ++r)
                    for (int c = 0; c < 3; ++c) t[c] += slots[r * 3 + c];
                const double Rk = (t[0] / (double)mu + t[1] / (double)tau - 2.0 * t[2]) * P.h * P.h;
                const int cv = Rk < P.tol;
                const int lt = (globaltimer() - t0) > P.budget_ns;
                const int stop = P.fixed || cv || lt || it >= cap;
                slots[48] = Rk;
                slots[49] = (double)(cv | (lt << 1) | (stop << 2));
            }
            cl.sync();
            R = slots0[48];
            const int d = (int)slots0[49];
            conv = d & 1;
            late = (d >> 1) & 1;
            if (d & 4) break;
        }
    }
    // write the level state back
    for (int idx = threadIdx.x; idx < nb; idx += T) {
        const size_t g = (size_t)jb * nx + idx;
        a.m1[g] = s1[idx];
        a.m2[g] = s2[idx];
        a.phi[g] = ph[idx];
    }
    if (rank == 0 && threadIdx.x == 0) {
        if (P.ctl) {
            P.ctl->iters[P.level] = it;
            P.ctl->fpr[P.level] = R;
            P.ctl->conv[P.level] = conv;
            if (late && !conv) P.ctl->timeout = 1;
        }
        if (P.fpr_out) *P.fpr_out = R;
        if (P.iters_out) *P.iters_out = it;
    }
    // keep every CTA's shared memory alive until the remote reads are done
    cl.sync();
}

template <int NORM>
static cudaError_t res_attr()
{
    cudaError_t e = cudaFuncSetAttribute(k_resident<NORM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)resident_smem(RES_MAX_NODES));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_resident<NORM>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

cudaError_t resident_prepare(int)
{
    cudaError_t e;
    if ((e = res_attr<W1_NORM_L1>()) != cudaSuccess) return e;
    return res_attr<W1_NORM_L2>();
}

static void resident_config(int norm, int cluster, int nx, int ny, cudaLaunchConfig_t& cfg, cudaLaunchAttribute* attr,
                            const void** fn)
{
    const int band = (ny / cluster) * nx;
    const int threads = band < RES_THREADS ? ((band + 31) / 32) * 32 : RES_THREADS;
    cfg = cudaLaunchConfig_t{};
    cfg.gridDim = dim3(cluster, 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = resident_smem(band);
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    *fn = norm == W1_NORM_L1 ? (const void*)k_resident<W1_NORM_L1> : (const void*)k_resident<W1_NORM_L2>;
}

int resident_cluster_ok(int norm, int cluster, int nx, int ny)
{
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    const void* fn = nullptr;
    resident_config(norm, cluster, nx, ny, cfg, attr, &fn);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

cudaError_t launch_resident(int norm, int cluster, const ResArgs& a, cudaStream_t s)
{
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    const void* fn = nullptr;
    resident_config(norm, cluster, a.it.nx, a.it.ny, cfg, attr, &fn);
    cfg.stream = s;
    void* args[1] = {(void*)&a};
    return cudaLaunchKernelExC(&cfg, fn, args);
}

// ---------------------------------------------------------------------------
// Final statistics: W1 = f(m), dual bound, residual, certified bracket
// ---------------------------------------------------------------------------

static constexpr int FIN_BLOCKS = 304, FIN_THREADS = 256;

size_t final_part_doubles() { return (size_t)FIN_BLOCKS * 5; }

template <int NORM>
__global__ void __launch_bounds__(FIN_THREADS) k_final_a(const float* __restrict__ m1, const float* __restrict__ m2,
                                                         const float* __restrict__ phi, const float* __restrict__ rho,
                                                         int nx, int ny, double h, double* __restrict__ q,
                                                         double* part)
{
    __shared__ double sh[32 * 4];
    double v[4] = {0.0, 0.0, 0.0, 0.0};  // f, dual, res_l1, rho_l1
    double gm = 0.0;
    const long long n = (long long)nx * ny;
    const double h2 = h * h;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(k / nx), i = (int)(k - (long long)j * nx);
        const double a1 = (i < nx - 1) ? (double)m1[k] : 0.0;
        const double a2 = (j < ny - 1) ? (double)m2[k] : 0.0;
        v[0] += (NORM == W1_NORM_L1 ? fabs(a1) + fabs(a2) : sqrt(a1 * a1 + a2 * a2)) * h2;
        const double p = phi[k], r = rho[k];
        v[1] -= p * r * h2;
        double d = a1 + a2;
        if (i > 0) d -= (double)m1[k - 1];
        if (j > 0) d -= (double)m2[k - nx];
        const double e = r - d / h;
        q[k] = e * h2;
        v[2] += fabs(e) * h2;
        v[3] += fabs(r) * h2;
        const double g1 = (i < nx - 1) ? ((double)phi[k + 1] - p) / h : 0.0;
        const double g2 = (j < ny - 1) ? ((double)phi[k + nx] - p) / h : 0.0;
        const double gq = (NORM == W1_NORM_L1) ? fmax(fabs(g1), fabs(g2)) : sqrt(g1 * g1 + g2 * g2);
        gm = fmax(gm, gq);
    }
    block_sum<4>(v, sh);
    // max over the block
    gm = warp_max(gm);
    __shared__ double shm[32];
    if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = gm;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) gm = fmax(gm, shm[w]);
        for (int c = 0; c < 4; ++c) part[blockIdx.x * 5 + c] = v[c];
        part[blockIdx.x * 5 + 4] = gm;
    }
}

// One block: sums the partials, then routes the residual masses q along the
// dyadic tree (each 2x2 block sends its masses to its first node; offsets
// (1,0), (0,1) cost one edge of the current spacing, (1,1) two), finishing
// with a diameter bound on the last grid.  This is an explicit flux carrying
// rho - div m, hence f + route >= W1 of the discrete problem.
__global__ void __launch_bounds__(1024) k_final_b(int nx, int ny, double h, double* q, double* q2,
                                                  const double* part, int nparts, Ctl* ctl)
{
    __shared__ double sh[32 * 4];
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    double gm = 0.0;
    for (int b = threadIdx.x; b < nparts; b += blockDim.x) {
        for (int c = 0; c < 4; ++c) v[c] += part[b * 5 + c];
        gm = fmax(gm, part[b * 5 + 4]);
    }
    block_sum<4>(v, sh);
    __shared__ double tot[4];
    if (threadIdx.x == 0)
        for (int c = 0; c < 4; ++c) tot[c] = v[c];
    gm = warp_max(gm);
    __shared__ double shm[32];
    if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = gm;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) gm = fmax(gm, shm[w]);

    int cx = nx, cy = ny;
    double hx = h, hy = h, cost = 0.0;
    double* src = q;
    double* dst = q2;
    for (;;) {
        const int px = (cx > 1 && (cx & 1) == 0), py = (cy > 1 && (cy & 1) == 0);
        const int stopx = (cx > 1 && (cx & 1)), stopy = (cy > 1 && (cy & 1));
        if (stopx || stopy || (!px && !py)) break;
        const int bx = px ? 2 : 1, by = py ? 2 : 1;
        const int ncx = cx / bx, ncy = cy / by;
        const long long nc = (long long)ncx * ncy;
        for (long long k = threadIdx.x; k < nc; k += blockDim.x) {
            const int J = (int)(k / ncx), I = (int)(k - (long long)J * ncx);
            double total = 0.0;
            for (int b = 0; b < by; ++b)
                for (int a = 0; a < bx; ++a) {
                    const double qa = src[(size_t)(by * J + b) * cx + (bx * I + a)];
                    cost += fabs(qa) * (a * hx + b * hy);
                    total += qa;
                }
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
    double pos = 0.0, neg = 0.0;
    for (long long k = threadIdx.x; k < (long long)cx * cy; k += blockDim.x) {
        const double x = src[k];
        if (x > 0) pos += x;
        else neg -= x;
    }
    double w[4] = {cost, pos, neg, 0.0};
    block_sum<4>(w, sh);
    if (threadIdx.x == 0) {
        const double diam = (cx - 1) * hx + (cy - 1) * hy;
        const double route = w[0] + diam * fmax(w[1], w[2]);
        ctl->f = tot[0];
        ctl->dual = tot[1];
        ctl->res_l1 = tot[2];
        ctl->rho_l1 = tot[3];
        ctl->gmax = gm;
        ctl->route = route;
        ctl->lb = tot[1] / fmax(1.0, gm);
        ctl->ub = tot[0] + route;
    }
}

cudaError_t launch_final(int norm, const float* m1, const float* m2, const float* phi, const float* rho, int nx,
                         int ny, double h, double* q, double* part, Ctl* ctl, cudaStream_t s)
{
    double* q2 = q + (size_t)nx * ny;
    if (norm == W1_NORM_L1)
        k_final_a<W1_NORM_L1><<<FIN_BLOCKS, FIN_THREADS, 0, s>>>(m1, m2, phi, rho, nx, ny, h, q, part);
    else
        k_final_a<W1_NORM_L2><<<FIN_BLOCKS, FIN_THREADS, 0, s>>>(m1, m2, phi, rho, nx, ny, h, q, part);
    k_final_b<<<1, 1024, 0, s>>>(nx, ny, h, q, q2, part, FIN_BLOCKS, ctl);
    return cudaGetLastError();
}

}  // namespace w1
