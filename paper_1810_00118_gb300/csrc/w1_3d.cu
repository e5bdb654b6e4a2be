// w1_3d.cu -- Algorithm 3 on three-dimensional grids (the paper's analysis is
// for general d; this is d = 3).
//
// Voxel-centre grid nx x ny x nz, arrays [nz][ny][nx] (x fastest), flux
// components m1, m2, m3 along x, y, z with zero flux through the boundary,
// inner products weighted by h^3.  A streamed step of eq. primaldual is one
// launch (k3_step: m' at each voxel and its lower neighbours, then phi', from
// the old state into other buffers) or two (k3_mprime: m' = prox_{mu||.||_p}
// (m + mu grad phi) in place and mbar = 2 m' - m; k3_phi: phi' = phi + tau
// (div mbar - rho) in place, + the terms of R^k).  A node's m' needs phi on
// three neighbours and its phi' needs mbar on three others: the two-launch step
// synchronises at the launch boundary, the one-launch step recomputes m' on the
// lower neighbours instead.  Every K-th step forms
// R^k of eq. pd_stop (FP32 terms and per-thread values, FP64 across blocks) and
// the host reads it to decide the level's stop, as in the eager mode of the 2-D
// plans.  Restriction (2x2x2 means), the voxel-centre Interpolate, prep and the
// certificates (f(m), the dual bound, the octree route bound) are kernels too.
// Levels of at most 4096 voxels per CTA (one CTA, or a cluster of z-slabs) run
// all their steps and stop tests in one launch on chip instead (k3_resident).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <cooperative_groups.h>

#include "w1_device.cuh"
#include "w1_internal.h"

namespace cg = cooperative_groups;

namespace w1 {

static constexpr int T3 = 256;

struct Dims3 {
    int nx, ny, nz;
    long long n;
};

__device__ __forceinline__ void node3(const Dims3& d, long long q, int& i, int& j, int& k)
{
    const long long plane = (long long)d.nx * d.ny;
    k = (int)(q / plane);
    const long long r = q - (long long)k * plane;
    j = (int)(r / d.nx);
    i = (int)(r - (long long)j * d.nx);
}

// Node-wise proximal map of mu ||.||_p on R^3.
template <int NORM>
__device__ __forceinline__ void prox3(const float v[3], float mu, float o[3])
{
    if (NORM == W1_NORM_L1) {
#pragma unroll
        for (int c = 0; c < 3; ++c) o[c] = v[c] - fminf(fmaxf(v[c], -mu), mu);
    } else if (NORM == W1_NORM_L2) {
        const float s = fmaxf(1.f - mu * rsqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]), 0.f);
#pragma unroll
        for (int c = 0; c < 3; ++c) o[c] = v[c] * s;
    } else {
        // v - mu Proj_{l1 ball}(v / mu): shrink the magnitudes by the threshold t of
        // the projection (sorted magnitudes s0 >= s1 >= s2)
        const float a0 = fabsf(v[0]), a1 = fabsf(v[1]), a2 = fabsf(v[2]);
        if (a0 + a1 + a2 <= mu) {  // v / mu inside the ball: the projection is v / mu, prox = 0
#pragma unroll
            for (int c = 0; c < 3; ++c) o[c] = 0.f;
            return;
        }
        float s0 = fmaxf(a0, fmaxf(a1, a2)), s2 = fminf(a0, fminf(a1, a2));
        float s1 = a0 + a1 + a2 - s0 - s2;
        // threshold on v / mu scaled by mu: largest r with s_r - (cum_r - mu) / (r + 1) > 0
        float t = s0 - mu;
        const float t1 = 0.5f * (s0 + s1 - mu);
        if (s1 - t1 > 0.f) t = t1;
        const float t2 = (s0 + s1 + s2 - mu) / 3.f;
        if (s2 - t2 > 0.f) t = t2;
        // projection p = sign(v) max(|v| - t, 0) / mu ; prox = v - mu p
        const float a[3] = {a0, a1, a2};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float pm = fmaxf(a[c] - t, 0.f);  // mu * |p_c|
            o[c] = copysignf(a[c] - pm, v[c]);
        }
    }
}

template <int NORM>
__global__ void __launch_bounds__(T3) k3_mprime(Dims3 d, float mu, float ih, float* __restrict__ m1,
                                                 float* __restrict__ m2, float* __restrict__ m3,
                                                 const float* __restrict__ phi, float* __restrict__ b1,
                                                 float* __restrict__ b2, float* __restrict__ b3)
{
    const long long q = (long long)blockIdx.x * T3 + threadIdx.x;
    if (q >= d.n) return;
    int i, j, k;
    node3(d, q, i, j, k);
    const float p = phi[q];
    const bool e1 = i < d.nx - 1, e2 = j < d.ny - 1, e3 = k < d.nz - 1;
    const float v[3] = {e1 ? fmaf(mu * ih, phi[q + 1] - p, m1[q]) : 0.f,
                        e2 ? fmaf(mu * ih, phi[q + d.nx] - p, m2[q]) : 0.f,
                        e3 ? fmaf(mu * ih, phi[q + (long long)d.nx * d.ny] - p, m3[q]) : 0.f};
    float o[3];
    prox3<NORM>(v, mu, o);
    if (!e1) o[0] = 0.f;
    if (!e2) o[1] = 0.f;
    if (!e3) o[2] = 0.f;
    b1[q] = 2.f * o[0] - m1[q];
    b2[q] = 2.f * o[1] - m2[q];
    b3[q] = 2.f * o[2] - m3[q];
    m1[q] = o[0];
    m2[q] = o[1];
    m3[q] = o[2];
}

// phi' = phi + tau (div mbar - rho); on a test step also R^k (dm = mbar - m').
template <bool CHECK>
__global__ void __launch_bounds__(T3) k3_phi(Dims3 d, float tau, float ih, double mu_d, double tau_d, double h,
                                              const float* __restrict__ rho, float* __restrict__ phi,
                                              const float* __restrict__ b1, const float* __restrict__ b2,
                                              const float* __restrict__ b3, const float* __restrict__ m1,
                                              const float* __restrict__ m2, const float* __restrict__ m3,
                                              double* part, unsigned int* counter, double* r_out)
{
    float sa = 0.f, sb = 0.f, sc = 0.f;
    // one voxel per thread; a test step runs on fewer blocks, its threads taking
    // several voxels (see check_grid3)
    auto voxel = [&](const long long q) {
        int i, j, k;
        node3(d, q, i, j, k);
        const long long sy = d.nx, sz = (long long)d.nx * d.ny;
        const float dv = (b1[q] - (i > 0 ? b1[q - 1] : 0.f)) + (b2[q] - (j > 0 ? b2[q - sy] : 0.f)) +
                         (b3[q] - (k > 0 ? b3[q - sz] : 0.f));
        const float dp = tau * fmaf(dv, ih, -rho[q]);
        phi[q] += dp;
        if (CHECK) {
            auto dm = [&](const float* b, const float* m, long long x) { return b[x] - m[x]; };
            const float d1 = dm(b1, m1, q), d2 = dm(b2, m2, q), d3 = dm(b3, m3, q);
            const float dd = (d1 - (i > 0 ? dm(b1, m1, q - 1) : 0.f)) + (d2 - (j > 0 ? dm(b2, m2, q - sy) : 0.f)) +
                             (d3 - (k > 0 ? dm(b3, m3, q - sz) : 0.f));
            sa += d1 * d1 + d2 * d2 + d3 * d3;
            sb += dp * dp;
            sc += dp * dd;  // h <dphi, div dm> before the 1/h
        }
    };
    if (CHECK) {
        for (long long q = (long long)blockIdx.x * T3 + threadIdx.x; q < d.n; q += (long long)gridDim.x * T3) voxel(q);
    } else {
        const long long q = (long long)blockIdx.x * T3 + threadIdx.x;
        if (q < d.n) voxel(q);
    }
    if (!CHECK) return;
    __shared__ double sh[64 * 3];
    __shared__ bool last;
    double v[3];
    ff_block_sum3(sa, sb, sc, reinterpret_cast<float*>(sh), v);
    if (threadIdx.x == 0) {
        part[blockIdx.x * 3 + 0] = v[0];
        part[blockIdx.x * 3 + 1] = v[1];
        part[blockIdx.x * 3 + 2] = v[2];
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    CSum t[3];
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
        for (int c = 0; c < 3; ++c) t[c].add(((volatile double*)part)[b * 3 + c]);
    block_csum<3>(t, sh);
    if (threadIdx.x == 0) {
        *r_out = (t[0].value() / mu_d + t[1].value() / tau_d - 2.0 * t[2].value() / h) * h * h * h;
        *counter = 0;
    }
}

// One step of eq. primaldual in one launch, for levels too large for the
// on-chip kernels.  Each thread forms m' at its voxel and at its three lower
// neighbours (recomputed there from the old state with k3_mprime's arithmetic),
// then div mbar (mbar = 2 m' - m) and phi' (k3_phi's arithmetic).  The old
// state is read and the new one written to other buffers, since neighbours
// read old values: DRAM moves m, phi and rho in and m', phi' out (36 B per
// voxel; the two-launch step moves 64 B).  The new state is bitwise the
// two-launch step's; R^k may differ in rounding (contraction of its sums).
template <int NORM, bool CHECK>
__global__ void __launch_bounds__(T3) k3_step(Dims3 d, float mu, float tau, float ih, double mu_d, double tau_d,
                                               double h, const float* __restrict__ rho,
                                               const float* __restrict__ m1, const float* __restrict__ m2,
                                               const float* __restrict__ m3, const float* __restrict__ phi,
                                               float* __restrict__ n1, float* __restrict__ n2,
                                               float* __restrict__ n3, float* __restrict__ nphi, double* part,
                                               unsigned int* counter, double* r_out)
{
    float sa = 0.f, sb = 0.f, sc = 0.f;
    // one voxel per thread; a test step runs on fewer blocks, its threads taking
    // several voxels (see check_grid3)
    auto voxel = [&](const long long q) {
        int i, j, k;
        node3(d, q, i, j, k);
        const long long sy = d.nx, sz = (long long)d.nx * d.ny;
        // m' at voxel x = (xi, xj, xk) (index x), as k3_mprime forms it
        auto mprime = [&](long long x, int xi, int xj, int xk, float (&o)[3]) {
            const float p = phi[x];
            const bool e1 = xi < d.nx - 1, e2 = xj < d.ny - 1, e3 = xk < d.nz - 1;
            const float v[3] = {e1 ? fmaf(mu * ih, phi[x + 1] - p, m1[x]) : 0.f,
                                e2 ? fmaf(mu * ih, phi[x + sy] - p, m2[x]) : 0.f,
                                e3 ? fmaf(mu * ih, phi[x + sz] - p, m3[x]) : 0.f};
            prox3<NORM>(v, mu, o);
            if (!e1) o[0] = 0.f;
            if (!e2) o[1] = 0.f;
            if (!e3) o[2] = 0.f;
        };
        float o[3];
        mprime(q, i, j, k, o);
        const float b1 = 2.f * o[0] - m1[q], b2 = 2.f * o[1] - m2[q], b3 = 2.f * o[2] - m3[q];
        // the lower neighbours' mbar component across the shared face (and dm there)
        float l1 = 0.f, l2 = 0.f, l3 = 0.f, e1 = 0.f, e2 = 0.f, e3 = 0.f;
        if (i > 0) {
            float t[3];
            mprime(q - 1, i - 1, j, k, t);
            l1 = 2.f * t[0] - m1[q - 1];
            e1 = l1 - t[0];
        }
        if (j > 0) {
            float t[3];
            mprime(q - sy, i, j - 1, k, t);
            l2 = 2.f * t[1] - m2[q - sy];
            e2 = l2 - t[1];
        }
        if (k > 0) {
            float t[3];
            mprime(q - sz, i, j, k - 1, t);
            l3 = 2.f * t[2] - m3[q - sz];
            e3 = l3 - t[2];
        }
        const float dv = (b1 - l1) + (b2 - l2) + (b3 - l3);
        const float p = phi[q];
        const float dp = tau * fmaf(dv, ih, -rho[q]);
        nphi[q] = p + dp;
        n1[q] = o[0];
        n2[q] = o[1];
        n3[q] = o[2];
        if (CHECK) {
            const float d1 = b1 - o[0], d2 = b2 - o[1], d3 = b3 - o[2];
            const float dd = (d1 - e1) + (d2 - e2) + (d3 - e3);
            sa += d1 * d1 + d2 * d2 + d3 * d3;
            sb += dp * dp;
            sc += dp * dd;  // h <dphi, div dm> before the 1/h
        }
    };
    if (CHECK) {
        for (long long q = (long long)blockIdx.x * T3 + threadIdx.x; q < d.n; q += (long long)gridDim.x * T3) voxel(q);
    } else {
        const long long q = (long long)blockIdx.x * T3 + threadIdx.x;
        if (q < d.n) voxel(q);
    }
    if (!CHECK) return;
    __shared__ double sh[64 * 3];
    __shared__ bool last;
    double v[3];
    ff_block_sum3(sa, sb, sc, reinterpret_cast<float*>(sh), v);
    if (threadIdx.x == 0) {
        part[blockIdx.x * 3 + 0] = v[0];
        part[blockIdx.x * 3 + 1] = v[1];
        part[blockIdx.x * 3 + 2] = v[2];
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    CSum t[3];
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
        for (int c = 0; c < 3; ++c) t[c].add(((volatile double*)part)[b * 3 + c]);
    block_csum<3>(t, sh);
    if (threadIdx.x == 0) {
        *r_out = (t[0].value() / mu_d + t[1].value() / tau_d - 2.0 * t[2].value() / h) * h * h * h;
        *counter = 0;
    }
}

__global__ void k3_restrict(Dims3 c, const float* __restrict__ f, float* __restrict__ out)
{
    const long long q = (long long)blockIdx.x * T3 + threadIdx.x;
    if (q >= c.n) return;
    int I, J, K;
    node3(c, q, I, J, K);
    const int nx = 2 * c.nx, ny = 2 * c.ny;
    float s = 0.f;
    for (int cz = 0; cz < 2; ++cz)
        for (int b = 0; b < 2; ++b) {
            const float* r = f + ((long long)(2 * K + cz) * ny + (2 * J + b)) * nx + 2 * I;
            s += r[0] + r[1];
        }
    out[q] = 0.125f * s;
}

__global__ void k3_prolong(Dims3 c, const float* __restrict__ m1c, const float* __restrict__ m2c,
                           const float* __restrict__ m3c, const float* __restrict__ phic, float* __restrict__ m1f,
                           float* __restrict__ m2f, float* __restrict__ m3f, float* __restrict__ phif)
{
    const Dims3 f{2 * c.nx, 2 * c.ny, 2 * c.nz, 8 * c.n};
    const long long q = (long long)blockIdx.x * T3 + threadIdx.x;
    if (q >= f.n) return;
    int i, j, k;
    node3(f, q, i, j, k);
    const int I = i >> 1, J = j >> 1, K = k >> 1;
    const int In = min(max((i & 1) ? I + 1 : I - 1, 0), c.nx - 1);
    const int Jn = min(max((j & 1) ? J + 1 : J - 1, 0), c.ny - 1);
    const int Kn = min(max((k & 1) ? K + 1 : K - 1, 0), c.nz - 1);
    auto C = [&](const float* a, int z, int y, int x) { return a[((long long)z * c.ny + y) * c.nx + x]; };
    float p = 0.f;
    for (int cz = 0; cz < 2; ++cz)
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) {
                const float w = (a ? 0.25f : 0.75f) * (b ? 0.25f : 0.75f) * (cz ? 0.25f : 0.75f);
                p += w * C(phic, cz ? Kn : K, b ? Jn : J, a ? In : I);
            }
    phif[q] = p;
    float v1 = (i & 1) ? C(m1c, K, J, I) : 0.5f * ((I > 0 ? C(m1c, K, J, I - 1) : 0.f) + C(m1c, K, J, I));
    float v2 = (j & 1) ? C(m2c, K, J, I) : 0.5f * ((J > 0 ? C(m2c, K, J - 1, I) : 0.f) + C(m2c, K, J, I));
    float v3 = (k & 1) ? C(m3c, K, J, I) : 0.5f * ((K > 0 ? C(m3c, K - 1, J, I) : 0.f) + C(m3c, K, J, I));
    m1f[q] = i == f.nx - 1 ? 0.f : v1;
    m2f[q] = j == f.ny - 1 ? 0.f : v2;
    m3f[q] = k == f.nz - 1 ? 0.f : v3;
}

// Certificates: per-block compensated FP64 partials (s, c) of sum ||m||_p,
// sum phi rho, sum |e|, sum |rho|, sum phi e (e = rho - div m; unscaled, h^3
// applied once at the end) and the first level of the route bound, and the
// maximum of the dual norm of grad phi (kept squared for p = 2, one square root
// per block).  When every side is even each thread takes a 2 x 2 x 2 cell: the
// non-negative terms of the cell are added in plain FP64 before their
// compensated sums, the masses of its voxels go to their cell's first voxel
// (an offset with s nonzero coordinates costs s h) and the cell's mass to q;
// otherwise q gets every voxel's mass.  1/h multiplies instead of dividing.
static constexpr int FIN3_PART = 13;
__host__ __device__ static inline bool final3_pooled(const Dims3& d)
{
    return d.nx % 2 == 0 && d.ny % 2 == 0 && d.nz % 2 == 0;
}
template <int NORM>
__global__ void __launch_bounds__(T3) k3_final_a(Dims3 d, double h, const float* __restrict__ m1,
                                                  const float* __restrict__ m2, const float* __restrict__ m3,
                                                  const float* __restrict__ phi, const float* __restrict__ rho,
                                                  double* __restrict__ q_out, double* part)
{
    const long long t = (long long)blockIdx.x * T3 + threadIdx.x;
    CSum v[6];
    double g = 0.0;
    const long long sy = d.nx, sz = (long long)d.nx * d.ny;
    const double inv_h = 1.0 / h, h3 = h * h * h;
    // the voxel's terms (non-negative ones into acc); returns its mass e h^3
    auto voxel = [&](int i, int j, int k, double (&acc)[3]) -> double {
        const long long q = k * sz + j * sy + i;
        const double a1 = fabs((double)m1[q]), a2 = fabs((double)m2[q]), a3 = fabs((double)m3[q]);
        acc[0] += NORM == W1_NORM_L1 ? __dadd_rn(__dadd_rn(a1, a2), a3)
                  : NORM == W1_NORM_L2 ? sqrt(__dadd_rn(__dadd_rn(__dmul_rn(a1, a1), __dmul_rn(a2, a2)), __dmul_rn(a3, a3)))
                                       : fmax(a1, fmax(a2, a3));
        const double p = phi[q], r = rho[q];
        v[1].add(__dmul_rn(p, r));
        const double dv = ((double)m1[q] * (i < d.nx - 1) - (i > 0 ? (double)m1[q - 1] : 0.0)) +
                          ((double)m2[q] * (j < d.ny - 1) - (j > 0 ? (double)m2[q - sy] : 0.0)) +
                          ((double)m3[q] * (k < d.nz - 1) - (k > 0 ? (double)m3[q - sz] : 0.0));
        const double e = __dsub_rn(r, __dmul_rn(dv, inv_h));
        acc[1] += fabs(e);
        acc[2] += fabs(r);
        v[4].add(__dmul_rn(p, e));
        const double g1 = i < d.nx - 1 ? fabs(((double)phi[q + 1] - p) * inv_h) : 0.0;
        const double g2 = j < d.ny - 1 ? fabs(((double)phi[q + sy] - p) * inv_h) : 0.0;
        const double g3 = k < d.nz - 1 ? fabs(((double)phi[q + sz] - p) * inv_h) : 0.0;
        g = fmax(g, NORM == W1_NORM_L1   ? fmax(g1, fmax(g2, g3))              // q = infinity
                    : NORM == W1_NORM_L2 ? g1 * g1 + g2 * g2 + g3 * g3 : g1 + g2 + g3);  // q = 2 (squared), q = 1
        return e * h3;
    };
    auto flush = [&](const double (&acc)[3]) {
        v[0].add(acc[0]);
        v[2].add(acc[1]);
        v[3].add(acc[2]);
    };
    if (final3_pooled(d)) {
        const int cx = d.nx / 2, cy = d.ny / 2;
        const long long cplane = (long long)cx * cy;
        if (t < d.n / 8) {
            const int K = (int)(t / cplane), r = (int)(t - K * cplane);
            const int J = r / cx, I = r - J * cx;
            double acc[3] = {0.0, 0.0, 0.0};
            double tot = 0.0, cost = 0.0;
            for (int zc = 0; zc < 2; ++zc)
                for (int b = 0; b < 2; ++b)
                    for (int a = 0; a < 2; ++a) {
                        const double qa = voxel(2 * I + a, 2 * J + b, 2 * K + zc, acc);
                        cost += fabs(qa) * (double)(a + b + zc);
                        tot += qa;
                    }
            flush(acc);
            v[5].add(__dmul_rn(cost, h));
            q_out[t] = tot;
        }
    } else if (t < d.n) {
        int i, j, k;
        node3(d, t, i, j, k);
        double acc[3] = {0.0, 0.0, 0.0};
        q_out[t] = voxel(i, j, k, acc);
        flush(acc);
    }
    __shared__ double sh[2 * 6 * T3];
    block_csum_sh<6>(v, sh);
    __shared__ double gm[32];
    g = warp_max(g);
    if ((threadIdx.x & 31) == 0) gm[threadIdx.x >> 5] = g;
    __syncthreads();
    if (threadIdx.x == 0) {
        double mx = 0.0;
        for (int w = 0; w < T3 / 32; ++w) mx = fmax(mx, gm[w]);
        for (int c = 0; c < 6; ++c) {
            part[blockIdx.x * FIN3_PART + 2 * c] = v[c].s;
            part[blockIdx.x * FIN3_PART + 2 * c + 1] = v[c].c;
        }
        part[blockIdx.x * FIN3_PART + 12] = NORM == W1_NORM_L2 ? sqrt(mx) : mx;
    }
}

struct Stats3Dev {
    double f, dual, res_l1, rho_l1, gmax, lb, route, ub, saddle;
};

// One block: the sums of the partials, then the dyadic route bound of the
// residual masses over the octree (the oracle's route bound): each pass sums
// 2x2x2 (or 2x2, 2) blocks into a compact coarser grid (ping-pong between q and
// q2), charging every mass the distance to its block's corner; the masses left
// on the last grid are charged its diameter.
__global__ void __launch_bounds__(T3) k3_final_b(Dims3 d, double h, const double* part, int nblk, double* q,
                                                  double* q2, Stats3Dev* out)
{
    __shared__ double sh[2 * 6 * T3];
    CSum t[6];
    double mx = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
        for (int c = 0; c < 6; ++c) {
            CSum x;
            x.s = part[b * FIN3_PART + 2 * c];
            x.c = part[b * FIN3_PART + 2 * c + 1];
            t[c].add(x);
        }
        mx = fmax(mx, part[b * FIN3_PART + 12]);
    }
    block_csum_sh<6>(t, sh);
    __shared__ double tot[5], sad;
    if (threadIdx.x == 0) {
        for (int c = 0; c < 5; ++c) tot[c] = t[c].value();
        CSum lag = t[0], pe;
        pe.s = -t[4].s;
        pe.c = -t[4].c;
        lag.add(pe);
        sad = lag.value();
    }
    __shared__ double gmx[32];
    mx = warp_max(mx);
    if ((threadIdx.x & 31) == 0) gmx[threadIdx.x >> 5] = mx;
    __syncthreads();
    // k3_final_a did the first level of the octree when every side is even
    // (its cost is t[5], valid in thread 0)
    double* src = q;
    double* dst = q2;
    const int pool = final3_pooled(d) ? 2 : 1;
    int cx = d.nx / pool, cy = d.ny / pool, cz = d.nz / pool;
    double hx = pool * h, hy = pool * h, hz = pool * h;
    CSum cost;
    for (;;) {
        const int px = cx > 1 && cx % 2 == 0, py = cy > 1 && cy % 2 == 0, pz = cz > 1 && cz % 2 == 0;
        const int odd = (cx > 1 && cx % 2) || (cy > 1 && cy % 2) || (cz > 1 && cz % 2);
        if (odd || (!px && !py && !pz)) break;
        const int bx = px ? 2 : 1, by = py ? 2 : 1, bz = pz ? 2 : 1;
        const int ncx = cx / bx, ncy = cy / by, ncz = cz / bz;
        const int cplane = ncx * ncy, cells = cplane * ncz;  // grids of up to 2^31 voxels
        for (int c = threadIdx.x; c < cells; c += blockDim.x) {
            const int K = c / cplane, r = c - K * cplane;
            const int J = r / ncx, I = r - J * ncx;
            double tot = 0.0, cs = 0.0;  // the block's costs are non-negative: one compensated add
            for (int zc = 0; zc < bz; ++zc)
                for (int b = 0; b < by; ++b)
                    for (int a = 0; a < bx; ++a) {
                        const double qa = src[((long long)(bz * K + zc) * cy + (by * J + b)) * cx + (bx * I + a)];
                        if (a | b | zc) cs += __dmul_rn(fabs(qa), (a ? hx : 0.0) + (b ? hy : 0.0) + (zc ? hz : 0.0));
                        tot += qa;
                    }
            cost.add(cs);
            dst[c] = tot;
        }
        __syncthreads();
        double* tmp = src;
        src = dst;
        dst = tmp;
        cx = ncx;
        cy = ncy;
        cz = ncz;
        if (px) hx *= 2.0;
        if (py) hy *= 2.0;
        if (pz) hz *= 2.0;
    }
    CSum pn[3];
    pn[0] = cost;
    if (threadIdx.x == 0) pn[0].add(t[5]);
    for (long long c = threadIdx.x; c < (long long)cx * cy * cz; c += blockDim.x) {
        const double v = src[c];
        if (v > 0) pn[1].add(v);
        else pn[2].add(-v);
    }
    block_csum_sh<3>(pn, sh);
    if (threadIdx.x == 0) {
        double g = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) g = fmax(g, gmx[w]);
        const double h3 = h * h * h;
        out->f = tot[0] * h3;
        out->dual = -tot[1] * h3;
        out->res_l1 = tot[2] * h3;
        out->rho_l1 = tot[3] * h3;
        out->saddle = sad * h3;
        out->gmax = g;
        out->lb = out->dual / fmax(1.0, g);
        out->route = pn[0].value() + ((cx - 1) * hx + (cy - 1) * hy + (cz - 1) * hz) * fmax(pn[1].value(), pn[2].value());
        out->ub = out->f + out->route;
    }
}

// ---------------------------------------------------------------------------
// On-chip level solve: every step of a level inside one launch
// ---------------------------------------------------------------------------
//
// A CTA (or a cluster of C CTAs, each holding a slab of nz / C planes) keeps
// its voxels' phi, m1, m2, m3 in shared memory for the neighbours to read; a
// thread owns four consecutive voxels of a row and keeps their m, phi, rho and
// D = h div m^k in registers.  One step is the 2-D on-chip step with a third
// axis: phase A forms m' from phi at x+1 (the next lane), y+1 (the row above)
// and z+1 (the plane above, or the halo plane pushed by the CTA above); phase B
// forms div m' from m1' at x-1, m2' at y-1 and m3' at z-1 (the plane below, or
// the halo plane pushed by the CTA below) and the dual step.  Halo planes move
// by st.async into the neighbour's shared memory, completing a transaction
// count on its mbarrier (the 2-D kernels' exchange with planes for rows).  The
// test step's cross term uses div dm = (D' - D) / h, already in registers.

static constexpr int R3_THREADS = 1024;
static constexpr int R3_MAX_NODES = 4 * R3_THREADS;  // voxels per CTA
static constexpr int R3_RED_BYTES = 1024;
static constexpr int R3_SLOT_BYTES = 512;
static constexpr unsigned long long R3_HALO_WAIT_NS = 200000000ull;

struct Res3 {
    long long iters;
    double fpr;
    int conv;
    int timeout;
};

struct R3Args {
    Dims3 d;
    float mu, tau, cm, ct;  // cm = mu / h, ct = tau / h
    double h, tol;
    int K, fixed;
    long long cap;
    unsigned long long budget_ns;
    const float* rho;
    float *m1, *m2, *m3, *phi;
    Res3* res;
};

static size_t r3_smem(int nb, int plane)
{
    return R3_RED_BYTES + R3_SLOT_BYTES + (size_t)nb * 4 * sizeof(float) + (size_t)2 * plane * sizeof(float);
}

static bool r3_fits(int nx, int ny, int nz, int C);

// The fewest CTAs with at most 4096 voxels each; else the most CTAs (the
// fastest step) with wide slabs of up to 16384.
static int r3_cluster_for(int nx, int ny, int nz)
{
    if (nx % 4 != 0) return 0;
    for (int c = 1; c <= 16; c *= 2)
        if (nz % c == 0 && (long long)(nz / c) * nx * ny <= R3_MAX_NODES) return c;
    for (int c = 16; c >= 1; c /= 2)
        if (r3_fits(nx, ny, nz, c)) return c;
    return 0;
}

template <int NORM, bool CL>
__global__ void __launch_bounds__(R3_THREADS, 1) k3_resident(R3Args a)
{
    int C = 1, rank = 0;
    if (CL) {
        cg::cluster_group cl = cg::this_cluster();
        C = (int)cl.num_blocks();
        rank = (int)cl.block_rank();
    }
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nx = a.d.nx, ny = a.d.ny, nz = a.d.nz;
    const int plane = nx * ny, P = nz / C, kb = rank * P, nb = P * plane;
    double* red = reinterpret_cast<double*>(smraw);
    double* slots = reinterpret_cast<double*>(smraw + R3_RED_BYTES);
    float* ph = reinterpret_cast<float*>(smraw + R3_RED_BYTES + R3_SLOT_BYTES);
    float* s1 = ph + nb;
    float* s2 = s1 + nb;
    float* s3 = s2 + nb;
    float* hphi = s3 + nb;     // phi of the plane above the slab (from CTA rank + 1)
    float* hm3 = hphi + plane;  // m3' of the plane below the slab (from CTA rank - 1)
    const uint32_t bar_phi = smem_u32(slots + 56), bar_m3 = smem_u32(slots + 57);
    const size_t off = (size_t)kb * plane;
    const float mu = a.mu, tau = a.tau, cm = a.cm, ct = a.ct;

    const int t = threadIdx.x, lane = t & 31, W = nx >> 2;
    const bool own = 4 * t < nb;
    const int id = own ? 4 * t : 0;
    const int kl = own ? id / plane : 0;
    const int rem = id - kl * plane;  // index within the plane
    const int jl = rem / nx, i0 = rem - jl * nx;
    const bool last_col = own && i0 + 4 == nx, top_row = jl == ny - 1, top_plane = kb + kl == nz - 1;
    const bool slab_top = own && kl == P - 1, slab_bot = own && kl == 0;
    const bool has_up = CL && rank + 1 < C, has_dn = CL && rank > 0;
    (void)W;
    float m1[4] = {0.f, 0.f, 0.f, 0.f}, m2[4] = {0.f, 0.f, 0.f, 0.f}, m3[4] = {0.f, 0.f, 0.f, 0.f};
    float pv[4] = {0.f, 0.f, 0.f, 0.f}, rv[4] = {0.f, 0.f, 0.f, 0.f}, Dv[4] = {0.f, 0.f, 0.f, 0.f};
    if (own) {
        float4 x1 = *reinterpret_cast<const float4*>(a.m1 + off + id);
        float4 x2 = *reinterpret_cast<const float4*>(a.m2 + off + id);
        float4 x3 = *reinterpret_cast<const float4*>(a.m3 + off + id);
        const float4 xp = *reinterpret_cast<const float4*>(a.phi + off + id);
        const float4 xr = *reinterpret_cast<const float4*>(a.rho + off + id);
        // the pinned entries (zero flux through the last face on each axis) are zero
        if (last_col) x1.w = 0.f;
        if (top_row) x2 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (top_plane) x3 = make_float4(0.f, 0.f, 0.f, 0.f);
        m1[0] = x1.x; m1[1] = x1.y; m1[2] = x1.z; m1[3] = x1.w;
        m2[0] = x2.x; m2[1] = x2.y; m2[2] = x2.z; m2[3] = x2.w;
        m3[0] = x3.x; m3[1] = x3.y; m3[2] = x3.z; m3[3] = x3.w;
        pv[0] = xp.x; pv[1] = xp.y; pv[2] = xp.z; pv[3] = xp.w;
        rv[0] = xr.x; rv[1] = xr.y; rv[2] = xr.z; rv[3] = xr.w;
        *reinterpret_cast<float4*>(ph + id) = xp;
        *reinterpret_cast<float4*>(s1 + id) = x1;
        *reinterpret_cast<float4*>(s2 + id) = x2;
        *reinterpret_cast<float4*>(s3 + id) = x3;
    }
    if (CL && t == 0) {
        mbar_init(bar_phi, 1);
        mbar_init(bar_m3, 1);
        if (has_up) mbar_expect(bar_phi, 4u * plane);
        if (has_dn) mbar_expect(bar_m3, 4u * plane);
        mbar_init_fence();
    }
    if (CL) cg::this_cluster().sync();
    else __syncthreads();
    uint32_t slots0 = smem_u32(slots);
    if (CL) slots0 = dsmem_map(smem_u32(slots), 0);
    // m3 of the plane below the voxel run (initial state: read from the CTA below)
    float4 b3 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (own) {
        if (kl > 0) b3 = *reinterpret_cast<const float4*>(s3 + id - plane);
        else if (has_dn) b3 = dsmem_ld4(dsmem_map(smem_u32(s3 + (P - 1) * plane + rem), rank - 1));
    }
    {  // D^0 = h div m^0
        const float ln = __shfl_up_sync(FULL, m1[3], 1);
        if (own) {
            const float l = i0 == 0 ? 0.f : (lane == 0 ? s1[id - 1] : ln);
            const float4 b2 = jl > 0 ? *reinterpret_cast<const float4*>(s2 + id - nx) : make_float4(0.f, 0.f, 0.f, 0.f);
            const float bb2[4] = {b2.x, b2.y, b2.z, b2.w}, bb3[4] = {b3.x, b3.y, b3.z, b3.w};
#pragma unroll
            for (int c = 0; c < 4; ++c) Dv[c] = (m1[c] - (c ? m1[c - 1] : l)) + (m2[c] - bb2[c]) + (m3[c] - bb3[c]);
        }
    }
    if (rank == 0 && t == 0) {
        reinterpret_cast<unsigned long long*>(slots)[50] = globaltimer();
        slots[48] = 0.0;
        slots[49] = 0.0;
        slots[51] = 0.0;
    }
    if (CL) cg::this_cluster().sync();
    else __syncthreads();
    // the initial phi of the bottom plane goes to the CTA below
    if (slab_bot && has_dn)
        st_async4(dsmem_map(smem_u32(hphi + rem), rank - 1), make_float4(pv[0], pv[1], pv[2], pv[3]),
                  dsmem_map(bar_phi, rank - 1));
    unsigned par = 0;
    bool sync_fail = false;
    auto halo_wait = [&](uint32_t bar) {
        if (!sync_fail && !mbar_wait(bar, par, R3_HALO_WAIT_NS)) {
            sync_fail = true;
            dsmem_st_f64(slots0 + 8u * 51, 1.0);
        }
    };
    const int t_top = ((P - 1) * plane) >> 2;  // first thread of the top plane: re-arms bar_phi
    int it = 0;
    const int cap = (int)min(a.cap, (long long)INT_MAX);
    int next = a.fixed ? cap : a.K;
    float sa = 0.f, sb = 0.f, sc = 0.f;
    auto one_step = [&](auto test) {
        constexpr bool check = decltype(test)::value;
        // ---- phase A: m' = prox(m + mu grad phi)
        const float rn = __shfl_down_sync(FULL, pv[0], 1);
        if (own) {
            float4 uy = make_float4(pv[0], pv[1], pv[2], pv[3]), uz = uy;
            if (!top_row) uy = *reinterpret_cast<const float4*>(ph + id + nx);
            if (!top_plane) {
                if (!CL || kl < P - 1) {
                    uz = *reinterpret_cast<const float4*>(ph + id + plane);
                } else {
                    halo_wait(bar_phi);
                    uz = *reinterpret_cast<const float4*>(hphi + rem);
                    if (t == t_top) mbar_expect(bar_phi, 4u * plane);
                }
            }
            const float right = last_col ? pv[3] : (lane == 31 ? ph[id + 4] : rn);
            const float py[4] = {uy.x, uy.y, uy.z, uy.w}, pz[4] = {uz.x, uz.y, uz.z, uz.w};
            float n1[4], n2[4], n3[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float pr = c < 3 ? pv[c + 1] : right;
                const float v[3] = {fmaf(cm, pr - pv[c], m1[c]), fmaf(cm, py[c] - pv[c], m2[c]),
                                    fmaf(cm, pz[c] - pv[c], m3[c])};
                float o[3];
                prox3<NORM>(v, mu, o);
                n1[c] = o[0];
                n2[c] = o[1];
                n3[c] = o[2];
            }
            if (last_col) n1[3] = 0.f;
            if (top_row) n2[0] = n2[1] = n2[2] = n2[3] = 0.f;
            if (top_plane) n3[0] = n3[1] = n3[2] = n3[3] = 0.f;
            if constexpr (check) {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float d1 = n1[c] - m1[c], d2 = n2[c] - m2[c], d3 = n3[c] - m3[c];
                    sa = fmaf(d1, d1, fmaf(d2, d2, fmaf(d3, d3, sa)));
                }
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                m1[c] = n1[c];
                m2[c] = n2[c];
                m3[c] = n3[c];
            }
            *reinterpret_cast<float4*>(s1 + id) = make_float4(n1[0], n1[1], n1[2], n1[3]);
            *reinterpret_cast<float4*>(s2 + id) = make_float4(n2[0], n2[1], n2[2], n2[3]);
            *reinterpret_cast<float4*>(s3 + id) = make_float4(n3[0], n3[1], n3[2], n3[3]);
            if (CL && slab_top && has_up)
                st_async4(dsmem_map(smem_u32(hm3 + rem), rank + 1), make_float4(n3[0], n3[1], n3[2], n3[3]),
                          dsmem_map(bar_m3, rank + 1));
        }
        __syncthreads();
        // ---- phase B: phi' = phi + tau (div(2m' - m) - rho)
        const float ln = __shfl_up_sync(FULL, m1[3], 1);
        if (own) {
            const float l = i0 == 0 ? 0.f : (lane == 0 ? s1[id - 1] : ln);
            const float4 b2 = jl > 0 ? *reinterpret_cast<const float4*>(s2 + id - nx) : make_float4(0.f, 0.f, 0.f, 0.f);
            float4 bz = make_float4(0.f, 0.f, 0.f, 0.f);
            if (kl > 0) {
                bz = *reinterpret_cast<const float4*>(s3 + id - plane);
            } else if (has_dn) {
                halo_wait(bar_m3);
                bz = *reinterpret_cast<const float4*>(hm3 + rem);
                if (t == 0) mbar_expect(bar_m3, 4u * plane);
            }
            const float bb2[4] = {b2.x, b2.y, b2.z, b2.w}, bb3[4] = {bz.x, bz.y, bz.z, bz.w};
            float pn[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float Dn = (m1[c] - (c ? m1[c - 1] : l)) + (m2[c] - bb2[c]) + (m3[c] - bb3[c]);
                pn[c] = fmaf(ct, fmaf(2.f, Dn, -Dv[c]), fmaf(-tau, rv[c], pv[c]));
                if constexpr (check) {
                    const float ep = pn[c] - pv[c];
                    sb = fmaf(ep, ep, sb);
                    sc = fmaf(ep, Dn - Dv[c], sc);  // h <dphi, div dm>, scaled below
                }
                Dv[c] = Dn;
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) pv[c] = pn[c];
            *reinterpret_cast<float4*>(ph + id) = make_float4(pn[0], pn[1], pn[2], pn[3]);
            if (CL && slab_bot && has_dn)
                st_async4(dsmem_map(smem_u32(hphi + rem), rank - 1), make_float4(pn[0], pn[1], pn[2], pn[3]),
                          dsmem_map(bar_phi, rank - 1));
        }
        par ^= 1u;
        __syncthreads();
    };
    while (it < cap) {
        const int plain = (next - 1 < cap ? next - 1 : cap) - it;
        for (int r = 0; r < plain; ++r) one_step(std::false_type{});
        it += plain;
        if (it >= cap) break;
        sa = sb = sc = 0.f;
        one_step(std::true_type{});
        ++it;
        next += a.K;
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
            const double h3 = a.h * a.h * a.h;
            const double Rk = (tt[0].value() / (double)mu + tt[1].value() / (double)tau - 2.0 * (tt[2].value() / a.h)) * h3;
            const int cv = Rk < a.tol && slots[51] == 0.0;
            const int lt = (globaltimer() - reinterpret_cast<const unsigned long long*>(slots)[50]) > a.budget_ns ||
                           slots[51] != 0.0;
            const int stop = a.fixed || cv || lt || it >= cap;
            slots[48] = Rk;
            slots[49] = (double)(cv | (lt << 1) | (stop << 2));
        }
        if (CL) cg::this_cluster().sync();
        else __syncthreads();
        if ((int)dsmem_ld_f64(slots0 + 8u * 49) & 4) break;
    }
    // the phi pushed by the CTA above after the last step has not been read
    if (CL && slab_top && has_up) halo_wait(bar_phi);
    if (own) {
        *reinterpret_cast<float4*>(a.m1 + off + id) = make_float4(m1[0], m1[1], m1[2], m1[3]);
        *reinterpret_cast<float4*>(a.m2 + off + id) = make_float4(m2[0], m2[1], m2[2], m2[3]);
        *reinterpret_cast<float4*>(a.m3 + off + id) = make_float4(m3[0], m3[1], m3[2], m3[3]);
        *reinterpret_cast<float4*>(a.phi + off + id) = make_float4(pv[0], pv[1], pv[2], pv[3]);
    }
    if (rank == 0 && t == 0) {
        const int dcs = (int)slots[49];
        a.res->iters = it;
        a.res->fpr = slots[48];
        a.res->conv = dcs & 1;
        a.res->timeout = ((dcs >> 1) & 1) && !(dcs & 1);
    }
    if (CL) cg::this_cluster().sync();
}


// Wide slabs (the 3-D counterpart of the 2-D wide bands): up to 16384 voxels
// per CTA, a thread owning four runs of four voxels (run r at voxel 4 (t + r T)
// of the slab).  Shared memory holds what neighbours read: phi, m2 and m3 of
// the slab, the last m1 of each warp's 128 voxels (the left neighbour of the
// next warp's lane 0), and two halo planes.  Each thread's own rho, D, phi and
// m1 live in tensor memory: 16 columns per run, 64 per warp in the warp's lane
// quarter, all 512 columns of the SM (allocated by warp 0, freed before exit).
static constexpr int R3W_RUNS = 4;
static constexpr int R3W_MAX_NODES = 4 * R3W_RUNS * R3_THREADS;  // 16384
static constexpr int R3W_MAX_PLANE = 4096;                       // halo planes of a cluster slab
static constexpr uint32_t R3W_TMEM_COLS = 512;

// floats of the per-warp m1 array, padded to 16 bytes so that the halo planes
// after it stay aligned for 16-byte accesses
__host__ __device__ constexpr int r3w_s1b_floats(int nb) { return ((nb / 128) + 3) & ~3; }

static size_t r3w_smem(int nb, int plane, bool cl)
{
    return R3_RED_BYTES + R3_SLOT_BYTES + (size_t)nb * 3 * sizeof(float) + (size_t)r3w_s1b_floats(nb) * sizeof(float) +
           (cl ? (size_t)2 * plane * sizeof(float) : 0);
}

template <int NORM, bool CL>
__global__ void __launch_bounds__(R3_THREADS, 1) k3_wide(R3Args a)
{
    int C = 1, rank = 0;
    if (CL) {
        cg::cluster_group cl = cg::this_cluster();
        C = (int)cl.num_blocks();
        rank = (int)cl.block_rank();
    }
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nx = a.d.nx, ny = a.d.ny, nz = a.d.nz;
    const int plane = nx * ny, P = nz / C, kb = rank * P, nb = P * plane;
    double* red = reinterpret_cast<double*>(smraw);
    double* slots = reinterpret_cast<double*>(smraw + R3_RED_BYTES);
    float* ph = reinterpret_cast<float*>(smraw + R3_RED_BYTES + R3_SLOT_BYTES);
    float* s2 = ph + nb;
    float* s3 = s2 + nb;
    float* s1b = s3 + nb;        // m1 of the last voxel of each warp's 128
    float* hphi = s1b + r3w_s1b_floats(nb);  // phi of the plane above the slab (from CTA rank + 1)
    float* hm3 = hphi + plane;   // m3' of the plane below the slab (from CTA rank - 1)
    const uint32_t bar_phi = smem_u32(slots + 56), bar_m3 = smem_u32(slots + 57);
    const size_t off = (size_t)kb * plane;
    const float mu = a.mu, tau = a.tau, cm = a.cm, ct = a.ct;
    const int t = threadIdx.x, T = blockDim.x, lane = t & 31;
    const bool has_up = CL && rank + 1 < C, has_dn = CL && rank > 0;

    // tensor memory
    if (t < 32) {
        tmem_alloc(smem_u32(slots + 58), R3W_TMEM_COLS);
    }
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const uint32_t tb = *reinterpret_cast<volatile uint32_t*>(slots + 58) + ((32u * ((t >> 5) & 3)) << 16) +
                        64u * (uint32_t)(t >> 7);
    // run r: rho at 16 r, D at 16 r + 4, phi at 16 r + 8, m1 at 16 r + 12

    // pk = (kl << 24) | (jl << 12) | (i0 >> 2) of the run's first voxel, or -1
    int pk[R3W_RUNS];
#pragma unroll
    for (int r = 0; r < R3W_RUNS; ++r) {
        const int id = 4 * (t + r * T);
        pk[r] = -1;
        if (id < nb) {
            const int kl = id / plane, rem = id - kl * plane, jl = rem / nx, i0 = rem - jl * nx;
            pk[r] = (kl << 24) | (jl << 12) | (i0 >> 2);
            float4 x1 = *reinterpret_cast<const float4*>(a.m1 + off + id);
            float4 x2 = *reinterpret_cast<const float4*>(a.m2 + off + id);
            float4 x3 = *reinterpret_cast<const float4*>(a.m3 + off + id);
            const float4 xp = *reinterpret_cast<const float4*>(a.phi + off + id);
            if (i0 + 4 == nx) x1.w = 0.f;
            if (jl == ny - 1) x2 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (kb + kl == nz - 1) x3 = make_float4(0.f, 0.f, 0.f, 0.f);
            *reinterpret_cast<float4*>(ph + id) = xp;
            *reinterpret_cast<float4*>(s2 + id) = x2;
            *reinterpret_cast<float4*>(s3 + id) = x3;
            if (lane == 31) s1b[id >> 7] = x1.w;
            tmem_st4(tb + 16u * r, __ldg(reinterpret_cast<const float4*>(a.rho + off + id)));
            tmem_st4(tb + 16u * r + 8u, xp);
            tmem_st4(tb + 16u * r + 12u, x1);
        }
    }
    tmem_wait_st();
    if (CL && t == 0) {
        mbar_init(bar_phi, 1);
        mbar_init(bar_m3, 1);
        if (has_up) mbar_expect(bar_phi, 4u * plane);
        if (has_dn) mbar_expect(bar_m3, 4u * plane);
        mbar_init_fence();
    }
    if (CL) cg::this_cluster().sync();
    else __syncthreads();
    uint32_t slots0 = smem_u32(slots);
    if (CL) slots0 = dsmem_map(smem_u32(slots), 0);
    unsigned par = 0;
    bool sync_fail = false;
    auto halo_wait = [&](uint32_t bar) {
        if (!sync_fail && !mbar_wait(bar, par, R3_HALO_WAIT_NS)) {
            sync_fail = true;
            dsmem_st_f64(slots0 + 8u * 51, 1.0);
        }
    };
    const int id_top = (P - 1) * plane;  // first voxel of the top plane: its owner re-arms bar_phi
    // h div m of run r (left: previous lane, or the previous warp's last m1;
    // below in y: the slab; below in z: the slab, the CTA below's top plane
    // (initial state) or the halo plane it pushed)
    auto divergence = [&](int r, const float4& m1, float out[4], auto halo) {
        const int kl = pk[r] >> 24, jl = (pk[r] >> 12) & 0xfff, i0 = (pk[r] & 0xfff) << 2;
        const int rem = jl * nx + i0, id = kl * plane + rem;
        const float ln = __shfl_up_sync(FULL, m1.w, 1);
        const float l = i0 == 0 ? 0.f : (lane == 0 ? s1b[(id >> 7) - 1] : ln);
        const float4 m2 = *reinterpret_cast<const float4*>(s2 + id);
        const float4 m3 = *reinterpret_cast<const float4*>(s3 + id);
        const float4 b2 = jl > 0 ? *reinterpret_cast<const float4*>(s2 + id - nx) : make_float4(0.f, 0.f, 0.f, 0.f);
        float4 b3 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (kl > 0) {
            b3 = *reinterpret_cast<const float4*>(s3 + id - plane);
        } else if (has_dn) {
            if constexpr (decltype(halo)::value) {
                halo_wait(bar_m3);
                b3 = *reinterpret_cast<const float4*>(hm3 + rem);
                if (t == 0 && r == 0 && !sync_fail) mbar_expect(bar_m3, 4u * plane);
            } else {
                b3 = dsmem_ld4(dsmem_map(smem_u32(s3 + (P - 1) * plane + rem), rank - 1));
            }
        }
        out[0] = (m1.x - l) + (m2.x - b2.x) + (m3.x - b3.x);
        out[1] = (m1.y - m1.x) + (m2.y - b2.y) + (m3.y - b3.y);
        out[2] = (m1.z - m1.y) + (m2.z - b2.z) + (m3.z - b3.z);
        out[3] = (m1.w - m1.z) + (m2.w - b2.w) + (m3.w - b3.w);
    };
#pragma unroll
    for (int r = 0; r < R3W_RUNS; ++r)
        if (pk[r] >= 0) {
            float d0[4];
            divergence(r, tmem_ld4(tb + 16u * r + 12u), d0, std::false_type{});
            tmem_st4(tb + 16u * r + 4u, make_float4(d0[0], d0[1], d0[2], d0[3]));
        }
    tmem_wait_st();
    if (rank == 0 && t == 0) {
        reinterpret_cast<unsigned long long*>(slots)[50] = globaltimer();
        slots[48] = 0.0;
        slots[49] = 0.0;
        slots[51] = 0.0;
    }
    if (CL) cg::this_cluster().sync();
    else __syncthreads();
    // the initial phi of the bottom plane goes to the CTA below
    if (has_dn) {
#pragma unroll
        for (int r = 0; r < R3W_RUNS; ++r)
            if (pk[r] >= 0 && (pk[r] >> 24) == 0) {
                const int rem = ((pk[r] >> 12) & 0xfff) * nx + ((pk[r] & 0xfff) << 2);
                st_async4(dsmem_map(smem_u32(hphi + rem), rank - 1), *reinterpret_cast<const float4*>(ph + rem),
                          dsmem_map(bar_phi, rank - 1));
            }
    }
    float sa = 0.f, sb = 0.f, sc = 0.f;
    auto wstep = [&](auto test) {
        constexpr bool check = decltype(test)::value;
        // ---- phase A: m' = prox(m + mu grad phi)
#pragma unroll
        for (int r = 0; r < R3W_RUNS; ++r) {
            if (pk[r] < 0) continue;
            const int kl = pk[r] >> 24, jl = (pk[r] >> 12) & 0xfff, i0 = (pk[r] & 0xfff) << 2;
            const int rem = jl * nx + i0, id = kl * plane + rem;
            const bool last_col = i0 + 4 == nx, top_row = jl == ny - 1, top_plane = kb + kl == nz - 1;
            const float4 p4 = tmem_ld4(tb + 16u * r + 8u);
            const float rn = __shfl_down_sync(FULL, p4.x, 1);
            const float4 a1 = tmem_ld4(tb + 16u * r + 12u);
            const float4 a2 = *reinterpret_cast<const float4*>(s2 + id);
            const float4 a3 = *reinterpret_cast<const float4*>(s3 + id);
            float4 uy = p4, uz = p4;
            if (!top_row) uy = *reinterpret_cast<const float4*>(ph + id + nx);
            if (!top_plane) {
                if (!CL || kl < P - 1) {
                    uz = *reinterpret_cast<const float4*>(ph + id + plane);
                } else {
                    halo_wait(bar_phi);
                    uz = *reinterpret_cast<const float4*>(hphi + rem);
                    if (id == id_top && !sync_fail) mbar_expect(bar_phi, 4u * plane);
                }
            }
            const float right = last_col ? p4.w : (lane == 31 ? ph[id + 4] : rn);
            const float pv[4] = {p4.x, p4.y, p4.z, p4.w}, py[4] = {uy.x, uy.y, uy.z, uy.w},
                        pz[4] = {uz.x, uz.y, uz.z, uz.w};
            const float m1[4] = {a1.x, a1.y, a1.z, a1.w}, m2[4] = {a2.x, a2.y, a2.z, a2.w},
                        m3[4] = {a3.x, a3.y, a3.z, a3.w};
            float n1[4], n2[4], n3[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float pr = c < 3 ? pv[c + 1] : right;
                const float v[3] = {fmaf(cm, pr - pv[c], m1[c]), fmaf(cm, py[c] - pv[c], m2[c]),
                                    fmaf(cm, pz[c] - pv[c], m3[c])};
                float o[3];
                prox3<NORM>(v, mu, o);
                n1[c] = o[0];
                n2[c] = o[1];
                n3[c] = o[2];
            }
            if (last_col) n1[3] = 0.f;
            if (top_row) n2[0] = n2[1] = n2[2] = n2[3] = 0.f;
            if (top_plane) n3[0] = n3[1] = n3[2] = n3[3] = 0.f;
            if constexpr (check) {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float d1 = n1[c] - m1[c], d2 = n2[c] - m2[c], d3 = n3[c] - m3[c];
                    sa = fmaf(d1, d1, fmaf(d2, d2, fmaf(d3, d3, sa)));
                }
            }
            tmem_st4(tb + 16u * r + 12u, make_float4(n1[0], n1[1], n1[2], n1[3]));
            if (lane == 31) s1b[id >> 7] = n1[3];
            *reinterpret_cast<float4*>(s2 + id) = make_float4(n2[0], n2[1], n2[2], n2[3]);
            *reinterpret_cast<float4*>(s3 + id) = make_float4(n3[0], n3[1], n3[2], n3[3]);
            if (has_up && kl == P - 1)
                st_async4(dsmem_map(smem_u32(hm3 + rem), rank + 1), make_float4(n3[0], n3[1], n3[2], n3[3]),
                          dsmem_map(bar_m3, rank + 1));
        }
        tmem_wait_st();
        __syncthreads();
        // ---- phase B: phi' = phi + tau (div(2m' - m) - rho)
#pragma unroll
        for (int r = 0; r < R3W_RUNS; ++r) {
            if (pk[r] < 0) continue;
            float Dn[4];
            divergence(r, tmem_ld4(tb + 16u * r + 12u), Dn, std::true_type{});
            const int kl = pk[r] >> 24, rem = ((pk[r] >> 12) & 0xfff) * nx + ((pk[r] & 0xfff) << 2);
            const int id = kl * plane + rem;
            const float4 r4 = tmem_ld4(tb + 16u * r), d4 = tmem_ld4(tb + 16u * r + 4u),
                         p4 = tmem_ld4(tb + 16u * r + 8u);
            const float pv[4] = {p4.x, p4.y, p4.z, p4.w}, rv[4] = {r4.x, r4.y, r4.z, r4.w},
                        Do[4] = {d4.x, d4.y, d4.z, d4.w};
            float pn[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                pn[c] = fmaf(ct, fmaf(2.f, Dn[c], -Do[c]), fmaf(-tau, rv[c], pv[c]));
                if constexpr (check) {
                    const float ep = pn[c] - pv[c];
                    sb = fmaf(ep, ep, sb);
                    sc = fmaf(ep, Dn[c] - Do[c], sc);
                }
            }
            tmem_st4(tb + 16u * r + 4u, make_float4(Dn[0], Dn[1], Dn[2], Dn[3]));
            tmem_st4(tb + 16u * r + 8u, make_float4(pn[0], pn[1], pn[2], pn[3]));
            *reinterpret_cast<float4*>(ph + id) = make_float4(pn[0], pn[1], pn[2], pn[3]);
            if (has_dn && kl == 0)
                st_async4(dsmem_map(smem_u32(hphi + rem), rank - 1), make_float4(pn[0], pn[1], pn[2], pn[3]),
                          dsmem_map(bar_phi, rank - 1));
        }
        tmem_wait_st();
        par ^= 1u;
        __syncthreads();
    };
    long long it = 0;
    const long long cap = a.cap;
    while (it < cap) {
        const bool check = a.fixed ? (it + 1 == cap) : ((it + 1) % a.K == 0);
        if (!check) {
            wstep(std::false_type{});
            ++it;
            continue;
        }
        sa = sb = sc = 0.f;
        wstep(std::true_type{});
        ++it;
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
            for (int q = 0; q < C; ++q)
                for (int c = 0; c < 3; ++c) tt[c].add(slots[q * 3 + c]);
            const double h3 = a.h * a.h * a.h;
            const double Rk = (tt[0].value() / (double)mu + tt[1].value() / (double)tau - 2.0 * (tt[2].value() / a.h)) * h3;
            const int cv = Rk < a.tol && slots[51] == 0.0;
            const int lt = (globaltimer() - reinterpret_cast<const unsigned long long*>(slots)[50]) > a.budget_ns ||
                           slots[51] != 0.0;
            const int stop = a.fixed || cv || lt || it >= cap;
            slots[48] = Rk;
            slots[49] = (double)(cv | (lt << 1) | (stop << 2));
        }
        if (CL) cg::this_cluster().sync();
        else __syncthreads();
        if ((int)dsmem_ld_f64(slots0 + 8u * 49) & 4) break;
    }
    // the phi pushed by the CTA above after the last step has not been read
    if (has_up) {
        bool top_run = false;
#pragma unroll
        for (int r = 0; r < R3W_RUNS; ++r) top_run |= pk[r] >= 0 && (pk[r] >> 24) == P - 1;
        if (top_run) halo_wait(bar_phi);
    }
#pragma unroll
    for (int r = 0; r < R3W_RUNS; ++r) {
        if (pk[r] < 0) continue;
        const int id = (pk[r] >> 24) * plane + ((pk[r] >> 12) & 0xfff) * nx + ((pk[r] & 0xfff) << 2);
        *reinterpret_cast<float4*>(a.m1 + off + id) = tmem_ld4(tb + 16u * r + 12u);
        *reinterpret_cast<float4*>(a.m2 + off + id) = *reinterpret_cast<const float4*>(s2 + id);
        *reinterpret_cast<float4*>(a.m3 + off + id) = *reinterpret_cast<const float4*>(s3 + id);
        *reinterpret_cast<float4*>(a.phi + off + id) = *reinterpret_cast<const float4*>(ph + id);
    }
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (t < 32) tmem_dealloc(*reinterpret_cast<volatile uint32_t*>(slots + 58), R3W_TMEM_COLS);
    if (rank == 0 && t == 0) {
        const int dcs = (int)slots[49];
        a.res->iters = it;
        a.res->fpr = slots[48];
        a.res->conv = dcs & 1;
        a.res->timeout = ((dcs >> 1) & 1) && !(dcs & 1);
    }
    if (CL) cg::this_cluster().sync();
}

template <int NORM>
static cudaError_t r3_attr()
{
    const int smem = (int)r3_smem(R3_MAX_NODES, R3_MAX_NODES);
    cudaError_t e = cudaFuncSetAttribute(k3_resident<NORM, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k3_resident<NORM, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k3_resident<NORM, true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    const int wsmem = (int)r3w_smem(R3W_MAX_NODES, R3W_MAX_PLANE, true);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k3_wide<NORM, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, wsmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k3_wide<NORM, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, wsmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k3_wide<NORM, true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

static const void* r3_fn(int norm, bool cl, bool wide)
{
    if (wide) {
        if (norm == W1_NORM_L1) return cl ? (const void*)k3_wide<W1_NORM_L1, true> : (const void*)k3_wide<W1_NORM_L1, false>;
        if (norm == W1_NORM_L2) return cl ? (const void*)k3_wide<W1_NORM_L2, true> : (const void*)k3_wide<W1_NORM_L2, false>;
        return cl ? (const void*)k3_wide<W1_NORM_LINF, true> : (const void*)k3_wide<W1_NORM_LINF, false>;
    }
    if (norm == W1_NORM_L1) return cl ? (const void*)k3_resident<W1_NORM_L1, true> : (const void*)k3_resident<W1_NORM_L1, false>;
    if (norm == W1_NORM_L2) return cl ? (const void*)k3_resident<W1_NORM_L2, true> : (const void*)k3_resident<W1_NORM_L2, false>;
    return cl ? (const void*)k3_resident<W1_NORM_LINF, true> : (const void*)k3_resident<W1_NORM_LINF, false>;
}

// A slab of nb voxels: the four-voxel layout up to 4096, the wide layout (tensor
// memory) up to 16384 when nb is a multiple of 128 and, in a cluster, the halo
// planes fit (plane <= 4096).
static bool r3_fits(int nx, int ny, int nz, int C)
{
    if (C < 1 || C > 16 || (C & (C - 1)) || nx % 4 || nz % C) return false;
    const long long nb = (long long)(nz / C) * nx * ny;
    if (nb <= R3_MAX_NODES) return true;
    return nb <= R3W_MAX_NODES && nb % 128 == 0 && (C == 1 || (long long)nx * ny <= R3W_MAX_PLANE) &&
           nx <= 4096 && ny <= 4096;
}

static bool r3_is_wide(const Dims3& d, int C) { return (long long)(d.nz / C) * d.nx * d.ny > R3_MAX_NODES; }

static void r3_config(const Dims3& d, int C, cudaLaunchConfig_t& cfg, cudaLaunchAttribute* attr)
{
    const int nb = (d.nz / C) * d.nx * d.ny;
    const bool wide = r3_is_wide(d, C);
    cfg = cudaLaunchConfig_t{};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(wide ? R3_THREADS : ((nb / 4 + 31) / 32) * 32, 1, 1);
    cfg.dynamicSmemBytes = wide ? r3w_smem(nb, d.nx * d.ny, C > 1) : r3_smem(nb, d.nx * d.ny);
    cfg.numAttrs = 0;
    if (C > 1) {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
}

// Cluster size for an on-chip 3-D level (0: the level does not fit, or the
// cluster cannot be placed on this device).
static int r3_choose(int norm, const Dims3& d, int want)
{
    const int C = want > 0 ? want : r3_cluster_for(d.nx, d.ny, d.nz);
    if (!r3_fits(d.nx, d.ny, d.nz, C)) return 0;
    if (r3_attr<W1_NORM_L1>() != cudaSuccess || r3_attr<W1_NORM_L2>() != cudaSuccess ||
        r3_attr<W1_NORM_LINF>() != cudaSuccess)
        return 0;
    if (C == 1) return 1;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    r3_config(d, C, cfg, attr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, r3_fn(norm, true, r3_is_wide(d, C)), &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n > 0 ? C : 0;
}

static cudaError_t r3_launch(int norm, int C, const R3Args& a, cudaStream_t s)
{
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    r3_config(a.d, C, cfg, attr);
    cfg.stream = s;
    void* args[1] = {const_cast<R3Args*>(&a)};
    return cudaLaunchKernelExC(&cfg, r3_fn(norm, C > 1, r3_is_wide(a.d, C)), args);
}

static dim3 grid3(long long n) { return dim3((unsigned)((n + T3 - 1) / T3)); }

static cudaError_t launch_mprime(int norm, const Dims3& d, float mu, float ih, float* m1, float* m2, float* m3,
                                 const float* phi, float* b1, float* b2, float* b3, cudaStream_t s)
{
    const dim3 g = grid3(d.n);
    if (norm == W1_NORM_L1) k3_mprime<W1_NORM_L1><<<g, T3, 0, s>>>(d, mu, ih, m1, m2, m3, phi, b1, b2, b3);
    else if (norm == W1_NORM_L2) k3_mprime<W1_NORM_L2><<<g, T3, 0, s>>>(d, mu, ih, m1, m2, m3, phi, b1, b2, b3);
    else k3_mprime<W1_NORM_LINF><<<g, T3, 0, s>>>(d, mu, ih, m1, m2, m3, phi, b1, b2, b3);
    return cudaGetLastError();
}

// Blocks of a test step: every block leaves FP64 partials that the last block
// adds up on one SM, where FP64 runs at a small fraction of the FP32 rate, so a
// test step runs on at most 8 blocks per SM (threads then take several voxels).
static unsigned check_grid3(long long n)
{
    int dev = 0, sms = 0;
    const unsigned full = grid3(n).x;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return full;
    }
    const unsigned cap = 8u * (unsigned)sms;
    return full < cap ? full : cap;
}

// Device scratch of a 3-D call: mbar planes, partials, counter, R^k, certificate.
struct Scratch3 {
    float* b = nullptr;      // 4 planes: mbar (two-launch step) or the other state (one-launch step)
    double* part = nullptr;  // FIN3_PART per block
    unsigned int* counter = nullptr;
    double* r = nullptr;
    double* q = nullptr;  // 2 planes of FP64 residual masses
    Stats3Dev* st = nullptr;
    Res3* res = nullptr;  // outcome of an on-chip level
    ~Scratch3()
    {
        cudaFree(res);
        cudaFree(b);
        cudaFree(part);
        cudaFree(counter);
        cudaFree(r);
        cudaFree(q);
        cudaFree(st);
    }
    cudaError_t alloc(long long n, bool certificate)
    {
        cudaError_t e = cudaMalloc(&b, 4 * n * sizeof(float));
        const long long blocks = (n + T3 - 1) / T3;
        if (e == cudaSuccess) e = cudaMalloc(&part, blocks * FIN3_PART * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&counter, sizeof(unsigned int));
        if (e == cudaSuccess) e = cudaMemset(counter, 0, sizeof(unsigned int));
        if (e == cudaSuccess) e = cudaMalloc(&r, sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&res, sizeof(Res3));
        if (e == cudaSuccess && certificate) e = cudaMalloc(&q, 2 * n * sizeof(double));
        if (e == cudaSuccess && certificate) e = cudaMalloc(&st, sizeof(Stats3Dev));
        return e;
    }
};

// `steps` steps on one level; the last one forms R^k into sc.r when test is set.
static cudaError_t steps3(int norm, const Dims3& d, double h, float mu, float tau, const float* rho, float* m1,
                          float* m2, float* m3, float* phi, long long steps, bool test, Scratch3& sc, cudaStream_t s)
{
    const float ih = (float)(1.0 / h);
    const long long n = d.n;
    float *b1 = sc.b, *b2 = sc.b + n, *b3 = sc.b + 2 * n;
    for (long long k = 0; k < steps; ++k) {
        cudaError_t e = launch_mprime(norm, d, mu, ih, m1, m2, m3, phi, b1, b2, b3, s);
        if (e != cudaSuccess) return e;
        if (test && k + 1 == steps)
            k3_phi<true><<<check_grid3(n), T3, 0, s>>>(d, tau, ih, mu, tau, h, rho, phi, b1, b2, b3, m1, m2, m3, sc.part,
                                                 sc.counter, sc.r);
        else
            k3_phi<false><<<grid3(n), T3, 0, s>>>(d, tau, ih, mu, tau, h, rho, phi, b1, b2, b3, m1, m2, m3, sc.part,
                                                  sc.counter, sc.r);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The same steps with one launch each (k3_step): the state alternates between
// (m1, m2, m3, phi) and the scratch planes, and ends in (m1, m2, m3, phi).
template <int NORM>
static cudaError_t steps3_one_norm(const Dims3& d, double h, float mu, float tau, const float* rho, float* m1,
                                   float* m2, float* m3, float* phi, long long steps, bool test, Scratch3& sc,
                                   cudaStream_t s)
{
    const float ih = (float)(1.0 / h);
    const long long n = d.n;
    float* A[4] = {m1, m2, m3, phi};
    float* B[4] = {sc.b, sc.b + n, sc.b + 2 * n, sc.b + 3 * n};
    for (long long k = 0; k < steps; ++k) {
        float** in = (k & 1) ? B : A;
        float** out = (k & 1) ? A : B;
        if (test && k + 1 == steps)
            k3_step<NORM, true><<<check_grid3(n), T3, 0, s>>>(d, mu, tau, ih, mu, tau, h, rho, in[0], in[1], in[2], in[3],
                                                        out[0], out[1], out[2], out[3], sc.part, sc.counter, sc.r);
        else
            k3_step<NORM, false><<<grid3(n), T3, 0, s>>>(d, mu, tau, ih, mu, tau, h, rho, in[0], in[1], in[2], in[3],
                                                         out[0], out[1], out[2], out[3], sc.part, sc.counter, sc.r);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (steps & 1)  // the last step wrote the scratch planes
        for (int c = 0; c < 4; ++c) {
            cudaError_t e = cudaMemcpyAsync(A[c], B[c], n * sizeof(float), cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

static cudaError_t steps3_one(int norm, const Dims3& d, double h, float mu, float tau, const float* rho, float* m1,
                              float* m2, float* m3, float* phi, long long steps, bool test, Scratch3& sc,
                              cudaStream_t s)
{
    if (norm == W1_NORM_L1) return steps3_one_norm<W1_NORM_L1>(d, h, mu, tau, rho, m1, m2, m3, phi, steps, test, sc, s);
    if (norm == W1_NORM_L2) return steps3_one_norm<W1_NORM_L2>(d, h, mu, tau, rho, m1, m2, m3, phi, steps, test, sc, s);
    return steps3_one_norm<W1_NORM_LINF>(d, h, mu, tau, rho, m1, m2, m3, phi, steps, test, sc, s);
}

static cudaError_t final3(int norm, const Dims3& d, double h, const float* m1, const float* m2, const float* m3,
                          const float* phi, const float* rho, Scratch3& sc, cudaStream_t s)
{
    const dim3 g = grid3(final3_pooled(d) ? d.n / 8 : d.n);
    if (norm == W1_NORM_L1) k3_final_a<W1_NORM_L1><<<g, T3, 0, s>>>(d, h, m1, m2, m3, phi, rho, sc.q, sc.part);
    else if (norm == W1_NORM_L2) k3_final_a<W1_NORM_L2><<<g, T3, 0, s>>>(d, h, m1, m2, m3, phi, rho, sc.q, sc.part);
    else k3_final_a<W1_NORM_LINF><<<g, T3, 0, s>>>(d, h, m1, m2, m3, phi, rho, sc.q, sc.part);
    k3_final_b<<<1, T3, 0, s>>>(d, h, sc.part, (int)g.x, sc.q, sc.q + d.n, sc.st);
    return cudaGetLastError();
}

}  // namespace w1

using namespace w1;

namespace {
thread_local std::string g_err3;
w1_status fail3(w1_status st, const std::string& m)
{
    g_err3 = m;
    return st;
}
#define W1_CK3(call)                                                                                \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) {                                                                    \
            cudaGetLastError();                                                                     \
            return fail3(e_ == cudaErrorMemoryAllocation ? W1_ERR_NOMEM : W1_ERR_CUDA,              \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                       \
        }                                                                                           \
    } while (0)
// Device workspace of w1_solve3d: the level arena, the step scratch and the
// control block, kept in a process-wide pool between calls (allocation and
// release cost milliseconds; concurrent callers each take their own).
struct Work3 {
    int device = -1;
    long long arena_floats = 0, n = 0;
    float* arena = nullptr;
    Scratch3 sc;
    Ctl* ctl = nullptr;
    double* part = nullptr;
    ~Work3()
    {
        cudaFree(arena);
        cudaFree(ctl);
        cudaFree(part);
    }
};
std::mutex g_pool_mu;
std::vector<Work3*> g_pool;

cudaError_t work3_acquire(int dev, long long arena_floats, long long n, Work3** out)
{
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        for (size_t k = 0; k < g_pool.size(); ++k) {
            Work3* w = g_pool[k];
            if (w->device == dev && w->arena_floats >= arena_floats && w->n >= n) {
                g_pool.erase(g_pool.begin() + (long)k);
                *out = w;
                return cudaSuccess;
            }
        }
    }
    auto* w = new (std::nothrow) Work3();
    if (!w) return cudaErrorMemoryAllocation;
    w->device = dev;
    w->arena_floats = arena_floats;
    w->n = n;
    cudaError_t e = cudaMalloc(&w->arena, arena_floats * sizeof(float));
    if (e == cudaSuccess) e = w->sc.alloc(n, true);
    if (e == cudaSuccess) e = cudaMalloc(&w->ctl, sizeof(Ctl));
    if (e == cudaSuccess) e = cudaMalloc(&w->part, prep_part_doubles(1) * sizeof(double));
    if (e != cudaSuccess) {
        delete w;
        return e;
    }
    *out = w;
    return cudaSuccess;
}

void work3_release(Work3* w)
{
    if (!w) return;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    g_pool.push_back(w);
}
}  // namespace

extern "C" void w1_3d_release_workspace(void)
{
    std::vector<Work3*> all;
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        all.swap(g_pool);
    }
    for (Work3* w : all) delete w;
}

extern "C" const char* w1_3d_last_error(void) { return g_err3.c_str(); }

extern "C" w1_status w1_cp_steps3d_ex(int nx, int ny, int nz, double h, int norm, float mu, float tau,
                                      const float* rho, float* m1, float* m2, float* m3, float* phi, long long iters,
                                      int path, int cluster, void* stream, double* fpr_last)
{
    if (nx < 1 || ny < 1 || nz < 1 || !(h > 0.0) || !rho || !m1 || !m2 || !m3 || !phi || iters < 0)
        return fail3(W1_ERR_INVALID_ARG, "bad arguments to w1_cp_steps3d");
    if (norm != W1_NORM_L1 && norm != W1_NORM_L2 && norm != W1_NORM_LINF)
        return fail3(W1_ERR_INVALID_ARG, "norm must be 1, 2 or 3");
    if (path < 1 || path > 3) return fail3(W1_ERR_INVALID_ARG, "path must be 1, 2 or 3");
    const Dims3 d{nx, ny, nz, (long long)nx * ny * nz};
    Scratch3 sc;
    W1_CK3(sc.alloc(d.n, false));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double r = 0.0;
    if (path == 1) {
        for (const void* q : {(const void*)rho, (const void*)m1, (const void*)m2, (const void*)m3, (const void*)phi})
            if (reinterpret_cast<uintptr_t>(q) % 16 != 0)
                return fail3(W1_ERR_INVALID_ARG, "the on-chip kernels need 16-byte aligned planes");
        const int C = r3_choose(norm, d, cluster);
        if (C == 0) return fail3(W1_ERR_UNSUPPORTED, "the level does not fit on chip with that cluster");
        if (iters > 0) {
            R3Args a{d, mu, tau, (float)(mu / h), (float)(tau / h), h, 0.0, (int)std::min(iters, (long long)INT_MAX),
                     1, iters, ~0ull, rho, m1, m2, m3, phi, sc.res};
            W1_CK3(r3_launch(norm, C, a, s));
            Res3 res{};
            W1_CK3(cudaMemcpyAsync(&res, sc.res, sizeof(res), cudaMemcpyDeviceToHost, s));
            W1_CK3(cudaStreamSynchronize(s));
            r = res.fpr;
        }
    } else {
        if (path == 2) W1_CK3(steps3(norm, d, h, mu, tau, rho, m1, m2, m3, phi, iters, true, sc, s));
        else W1_CK3(steps3_one(norm, d, h, mu, tau, rho, m1, m2, m3, phi, iters, true, sc, s));
        if (iters > 0) W1_CK3(cudaMemcpyAsync(&r, sc.r, sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    W1_CK3(cudaStreamSynchronize(s));
    if (fpr_last) *fpr_last = r;
    return W1_OK;
}

extern "C" w1_status w1_cp_steps3d(int nx, int ny, int nz, double h, int norm, float mu, float tau, const float* rho,
                                   float* m1, float* m2, float* m3, float* phi, long long iters, void* stream,
                                   double* fpr_last)
{
    return w1_cp_steps3d_ex(nx, ny, nz, h, norm, mu, tau, rho, m1, m2, m3, phi, iters, 2, 0, stream, fpr_last);
}

extern "C" w1_status w1_restrict3d(int nx, int ny, int nz, const float* fine, float* coarse, void* stream)
{
    if (nx < 2 || ny < 2 || nz < 2 || nx % 2 || ny % 2 || nz % 2 || !fine || !coarse)
        return fail3(W1_ERR_SHAPE, "w1_restrict3d needs even nx, ny, nz");
    const Dims3 c{nx / 2, ny / 2, nz / 2, (long long)(nx / 2) * (ny / 2) * (nz / 2)};
    k3_restrict<<<grid3(c.n), T3, 0, static_cast<cudaStream_t>(stream)>>>(c, fine, coarse);
    W1_CK3(cudaGetLastError());
    return W1_OK;
}

extern "C" w1_status w1_prolong3d(int ncx, int ncy, int ncz, const float* m1c, const float* m2c, const float* m3c,
                                  const float* phic, float* m1f, float* m2f, float* m3f, float* phif, void* stream)
{
    if (ncx < 1 || ncy < 1 || ncz < 1 || !m1c || !m2c || !m3c || !phic || !m1f || !m2f || !m3f || !phif)
        return fail3(W1_ERR_INVALID_ARG, "bad arguments to w1_prolong3d");
    const Dims3 c{ncx, ncy, ncz, (long long)ncx * ncy * ncz};
    k3_prolong<<<grid3(8 * c.n), T3, 0, static_cast<cudaStream_t>(stream)>>>(c, m1c, m2c, m3c, phic, m1f, m2f, m3f,
                                                                           phif);
    W1_CK3(cudaGetLastError());
    return W1_OK;
}

extern "C" w1_status w1_solve3d(int nx, int ny, int nz, double h, int levels, int norm, double tol,
                                const w1_options* opt, const float* rho0, const float* rho1, void* stream,
                                double* dist, float* flux, float* potential, w1_stats* stats)
{
    if (nx < 1 || ny < 1 || nz < 1 || !rho0 || !rho1 || !dist) return fail3(W1_ERR_INVALID_ARG, "bad arguments");
    if (norm != W1_NORM_L1 && norm != W1_NORM_L2 && norm != W1_NORM_LINF)
        return fail3(W1_ERR_INVALID_ARG, "norm must be 1, 2 or 3");
    w1_options o;
    w1_default_options(&o);
    if (opt) o = *opt;
    const int K = o.check_every > 0 ? o.check_every : 32;
    if (K < 1 || !(o.theta > 0.0) || o.theta > 1.0 || o.max_iters < 1 || o.path < 0 || o.path > 3)
        return fail3(W1_ERR_INVALID_ARG, "bad options");
    if (!(h > 0.0)) h = 1.0 / (double)std::max(nx, std::max(ny, nz));
    if (levels <= 0) {  // the paper's L = log2(1/h) - 3, kept divisible, coarsest side >= 2
        int L = (int)std::lround(std::log2(1.0 / h)) - 3;
        if (L < 1) L = 1;
        while (L > 1 && ((nx % (1 << (L - 1))) || (ny % (1 << (L - 1))) || (nz % (1 << (L - 1))) ||
                         (nx >> (L - 1)) < 2 || (ny >> (L - 1)) < 2 || (nz >> (L - 1)) < 2))
            --L;
        levels = L;
    }
    if (levels > W1_MAX_LEVELS) return fail3(W1_ERR_SHAPE, "at most 16 levels");
    const int div = 1 << (levels - 1);
    if (nx % div || ny % div || nz % div) return fail3(W1_ERR_SHAPE, "nx, ny, nz must be divisible by 2^(levels-1)");
    if (!(tol > 0.0)) tol = 1e-6 / 128.0 * (512.0 * h) * (512.0 * h);  // eq. stop_tol's 2-D formula (reading)
    int dev = 0;
    W1_CK3(cudaGetDevice(&dev));
    W1_CK3(resident_prepare(dev));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long n = (long long)nx * ny * nz;
    // per level: rho, m1, m2, m3, phi
    // per level: rho, m1, m2, m3, phi, each plane padded to 16 bytes so that every
    // plane of every level is aligned for the kernels' 16-byte accesses
    auto plane_stride = [&](int l) {
        const int sh = levels - 1 - l;
        return (((long long)(nx >> sh) * (ny >> sh) * (nz >> sh)) + 3) & ~3LL;
    };
    std::vector<long long> off(levels + 1, 0);
    for (int l = 0; l < levels; ++l) off[l + 1] = off[l] + 5 * plane_stride(l);
    // device workspace from the pool (kept between calls; w1_3d_release_workspace frees it)
    Work3* w = nullptr;
    W1_CK3(work3_acquire(dev, off[levels], n, &w));
    struct Back {
        Work3* w;
        ~Back() { work3_release(w); }
    } back{w};
    float* arena = w->arena;
    Scratch3& sc = w->sc;
    Ctl* ctl = w->ctl;
    double* part = w->part;
    W1_CK3(cudaMemsetAsync(ctl, 0, sizeof(Ctl), s));
    W1_CK3(cudaMemsetAsync(sc.counter, 0, sizeof(unsigned int), s));
    auto lvl = [&](int l, int c) { return arena + off[l] + c * plane_stride(l); };
    // prep (masses with h^3 weights: the prep kernel weights by h_2d^2, so pass h^(3/2))
    W1_CK3(launch_prep(rho0, rho1, n, 1, 1, std::pow(h, 1.5), ctl, part, lvl(levels - 1, 0), s));
    Ctl host{};
    W1_CK3(cudaMemcpyAsync(&host, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    W1_CK3(cudaStreamSynchronize(s));
    if (host.error) {
        *dist = NAN;
        return fail3(W1_ERR_MASS, "densities have different mass or a non-finite value");
    }
    for (int l = levels - 1; l > 0; --l) {
        const int sh = levels - 1 - l;
        const Dims3 c{(nx >> sh) / 2, (ny >> sh) / 2, (nz >> sh) / 2, 0};
        const Dims3 cc{c.nx, c.ny, c.nz, (long long)c.nx * c.ny * c.nz};
        k3_restrict<<<grid3(cc.n), T3, 0, s>>>(cc, lvl(l, 0), lvl(l - 1, 0));
    }
    W1_CK3(cudaGetLastError());
    w1_status ret = W1_OK;
    if (stats) std::memset(stats, 0, sizeof(*stats));
    bool all_conv = true, late_any = false;
    for (int l = 0; l < levels; ++l) {
        const int sh = levels - 1 - l;
        const Dims3 d{nx >> sh, ny >> sh, nz >> sh, (long long)(nx >> sh) * (ny >> sh) * (nz >> sh)};
        const double hl = h * (double)(1 << sh);
        const float mu = (float)(o.theta * hl / (2.0 * std::sqrt(3.0)));  // theta / ||A_h||, ||A_h|| <= 2 sqrt(3) / h
        const double tl = tol * std::pow(hl / h, o.alpha);
        if (l == 0) {
            W1_CK3(cudaMemsetAsync(lvl(0, 1), 0, 4 * plane_stride(0) * sizeof(float), s));
        } else {
            const Dims3 c{d.nx / 2, d.ny / 2, d.nz / 2, d.n / 8};
            k3_prolong<<<grid3(d.n), T3, 0, s>>>(c, lvl(l - 1, 1), lvl(l - 1, 2), lvl(l - 1, 3), lvl(l - 1, 4),
                                                 lvl(l, 1), lvl(l, 2), lvl(l, 3), lvl(l, 4));
            W1_CK3(cudaGetLastError());
        }
        NvtxRange range("w1 3-D level %d %dx%dx%d", l, d.nx, d.ny, d.nz);
        long long it = 0;
        double r = 0.0;
        bool conv = false, late = false;
        // on chip where the level fits (path 0 or 1); else one launch per step
        // (path 0 or 3), or two (path 2)
        const int C = (o.path == 0 || o.path == 1) ? r3_choose(norm, d, 0) : 0;
        if (o.path == 1 && C == 0) return fail3(W1_ERR_UNSUPPORTED, "a level does not fit on chip");
        if (late_any) {
            // a coarser level ran out of time: carry the state up without steps
        } else if (C > 0) {
            const unsigned long long budget =
                o.time_budget_s >= 1e9 ? ~0ull : (unsigned long long)(o.time_budget_s * 1e9);
            R3Args a{d, mu, mu, (float)(mu / hl), (float)(mu / hl), hl, tl, K, 0, o.max_iters, budget,
                     lvl(l, 0), lvl(l, 1), lvl(l, 2), lvl(l, 3), lvl(l, 4), sc.res};
            W1_CK3(r3_launch(norm, C, a, s));
            Res3 res{};
            W1_CK3(cudaMemcpyAsync(&res, sc.res, sizeof(res), cudaMemcpyDeviceToHost, s));
            W1_CK3(cudaStreamSynchronize(s));
            it = res.iters;
            r = res.fpr;
            conv = res.conv != 0;
            late = res.timeout != 0;
        } else {
            const auto t0 = std::chrono::steady_clock::now();
            while (it < o.max_iters) {
                if (o.path == 2)
                    W1_CK3(steps3(norm, d, hl, mu, mu, lvl(l, 0), lvl(l, 1), lvl(l, 2), lvl(l, 3), lvl(l, 4), K, true,
                                  sc, s));
                else
                    W1_CK3(steps3_one(norm, d, hl, mu, mu, lvl(l, 0), lvl(l, 1), lvl(l, 2), lvl(l, 3), lvl(l, 4), K,
                                      true, sc, s));
                it += K;
                W1_CK3(cudaMemcpyAsync(&r, sc.r, sizeof(double), cudaMemcpyDeviceToHost, s));
                W1_CK3(cudaStreamSynchronize(s));
                if (r < tl) {
                    conv = true;
                    break;
                }
                const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
                if (el > o.time_budget_s) {
                    late = true;
                    break;
                }
            }
        }
        if (stats && l < W1_MAX_LEVELS) {
            stats->nx[l] = d.nx;
            stats->ny[l] = d.ny;
            stats->iters[l] = it;
            stats->fpr[l] = r;
            stats->tol[l] = tl;
            stats->path[l] = C > 0 ? 1 : (o.path == 2 ? 2 : 3);  // on chip, two launches, one launch per step
            stats->cluster[l] = C;
        }
        all_conv &= conv;
        if (late && !late_any) {
            late_any = true;
            ret = fail3(W1_ERR_TIMEOUT, "the time budget ran out");
        }
        if (!conv && ret == W1_OK) ret = fail3(W1_ERR_NOT_CONVERGED, "a level hit max_iters");
    }
    const int L = levels;
    W1_CK3(final3(norm, Dims3{nx, ny, nz, n}, h, lvl(L - 1, 1), lvl(L - 1, 2), lvl(L - 1, 3), lvl(L - 1, 4),
                  lvl(L - 1, 0), sc, s));
    Stats3Dev st{};
    W1_CK3(cudaMemcpyAsync(&st, sc.st, sizeof(st), cudaMemcpyDeviceToHost, s));
    if (flux) {
        for (int c = 0; c < 3; ++c)
            W1_CK3(cudaMemcpyAsync(flux + c * n, lvl(L - 1, 1 + c), n * sizeof(float), cudaMemcpyDeviceToDevice, s));
    }
    if (potential) W1_CK3(cudaMemcpyAsync(potential, lvl(L - 1, 4), n * sizeof(float), cudaMemcpyDeviceToDevice, s));
    W1_CK3(cudaStreamSynchronize(s));
    *dist = o.estimate == 1 ? st.f : st.saddle;
    if (stats) {
        stats->levels = L;
        stats->w1 = *dist;
        stats->primal = st.f;
        stats->saddle = st.saddle;
        stats->dual = st.dual;
        stats->lb = st.lb;
        stats->ub = st.ub;
        stats->route = st.route;
        stats->res_l1 = st.res_l1;
        stats->rho_l1 = st.rho_l1;
        stats->gmax = st.gmax;
        stats->mass0 = host.mass0;
        stats->mass1 = host.mass1;
        stats->mass_shift = host.mean;
        stats->converged = all_conv && ret == W1_OK;
    }
    return ret;
}
