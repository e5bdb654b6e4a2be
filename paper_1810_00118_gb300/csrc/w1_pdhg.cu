// w1_pdhg.cu -- prox-PDHG kernels (Algorithm 2, and Algorithm 4 through the
// plan's level sequence).
//
// One step of eq. pdhg, with A = div^h, A^* = -grad and the zero-flux boundary:
//   v      = m - mu phibar                          (pinned entries zero)
//   psi    = (A A^*)^{-1} (div v - rho)             Neumann Poisson solve
//   m'     = v + grad psi                           (= Proj_{A m = rho}(v))
//   phi'   = Proj_{||.||_q <= 1}(phi + tau m')      node-wise
//   phibar = 2 phi' - phi
// A A^* = -div grad is the 5-point Neumann Laplacian; on this pixel-centre grid
// it is diagonal in the DCT-II basis with eigenvalues
//   (2 - 2 cos(pi kx / nx)) / h^2 + (2 - 2 cos(pi ky / ny)) / h^2,
// so the solve is DCT-II along rows, DCT-II along columns, a division, and the
// two inverse transforms.  Each DCT of length n (a power of two, <= 1024) is
// one complex FFT of length n of the reordered row (even samples ascending,
// odd samples descending) and a quarter-wave rotation; the inverse runs the
// same steps backwards.  Launches per step:
//   k_pd_resid  r = div v - rho                                  (stencil)
//   k_pd_rows<FWD_T>    DCT-II of each row, written transposed
//   k_pd_rows<SOLVE_T>  DCT-II of each column, / eigenvalue, DCT-III, written back
//   k_pd_rows<INV>      DCT-III of each row: psi
//   k_pd_update m', phi', phibar (+ the stop test G^k of eq. pdhg_stop)
// Rows are transformed in shared memory, 8 or more rows per CTA so that the
// transposed writes move whole 32-byte sectors.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "w1_device.cuh"
#include "w1_internal.h"

namespace w1 {

static constexpr int PD_TW = 4096;   // twiddle table: e^{-2 pi i k / 4096}, k < 4096
static constexpr int PD_MAXN = 1024;  // longest transform
static constexpr int PD_THREADS = 256;

static int ilog2(int n)
{
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

bool pd_level_ok(int nx, int ny)
{
    auto pow2 = [](int n) { return n >= 2 && n <= PD_MAXN && (n & (n - 1)) == 0; };
    return pow2(nx) && pow2(ny);
}

void pd_twiddles(float2* host)
{
    for (int k = 0; k < PD_TW; ++k) {
        const double a = 2.0 * 3.14159265358979323846 * (double)k / (double)PD_TW;
        host[k] = make_float2((float)std::cos(a), (float)-std::sin(a));
    }
}

void pd_eigen(int n, double h, float* host)
{
    for (int k = 0; k < n; ++k) host[k] = (float)((2.0 - 2.0 * std::cos(3.14159265358979323846 * k / n)) / (h * h));
}

size_t pd_twiddle_count() { return PD_TW; }

// rows per CTA: one butterfly per thread and stage, and at least 8 (32-byte sectors)
__host__ __device__ constexpr int pd_rows_per_cta(int n) { return 2 * PD_THREADS / n < 8 ? 8 : 2 * PD_THREADS / n; }

static size_t pd_rows_smem(int n)
{
    const int R = pd_rows_per_cta(n);
    // complex row buffer + padded real staging (spectrum, transposed write-out)
    return (size_t)R * n * sizeof(float2) + (size_t)R * (n + 1) * sizeof(float);
}

__device__ __forceinline__ int bitrev(int i, int logn) { return (int)(__brev((unsigned)i) >> (32 - logn)); }

// In-place radix-2 decimation-in-time FFT of R rows of n complex values stored
// in bit-reversed order (row r at buf + r n).  inv: conjugate twiddles (no 1/n).
__device__ void fft_rows(float2* buf, int n, int logn, int R, bool inv, const float2* __restrict__ tw)
{
    const int half = n >> 1, total = R * half;
    for (int s = 1; s <= logn; ++s) {
        const int hl = 1 << (s - 1), tstride = PD_TW >> s;
        for (int b = threadIdx.x; b < total; b += blockDim.x) {
            const int r = b >> (logn - 1), j = b & (half - 1);
            const int pos = j & (hl - 1), grp = j >> (s - 1);
            const int i0 = r * n + (grp << s) + pos, i1 = i0 + hl;
            float2 w = __ldg(tw + pos * tstride);
            if (inv) w.y = -w.y;
            const float2 a = buf[i0], c = buf[i1];
            const float2 t = make_float2(w.x * c.x - w.y * c.y, w.x * c.y + w.y * c.x);
            buf[i0] = make_float2(a.x + t.x, a.y + t.y);
            buf[i1] = make_float2(a.x - t.x, a.y - t.y);
        }
        __syncthreads();
    }
}

struct PdRowArgs {
    const float* in;   // pair 0: [nrows][n]
    float* out;        // pair 0: [n][nrows] (transposed modes) or [nrows][n]
    int n, logn, nrows;
    long long stride;  // elements between pairs
    const float2* tw;
    const float* lam_row;  // SOLVE_T: eigenvalue part of the row index (length nrows)
    const float* lam_pos;  // SOLVE_T: eigenvalue part of the position (length n)
    float scale;           // INV: output = scale * x
    const Ctl* ctl;
    int use_cond;
};

enum { PD_FWD_T = 0, PD_SOLVE_T = 1, PD_INV = 2 };

// DCT-II of the rows held (reordered, bit-reversed) in buf -> spectrum X in xs (padded rows).
__device__ void dct2_finish(const float2* buf, float* xs, int n, int R, const float2* __restrict__ tw)
{
    const int step = PD_TW / (4 * n);  // e^{-i pi k / (2n)} = tw[k step]
    for (int e = threadIdx.x; e < R * n; e += blockDim.x) {
        const int r = e / n, k = e - r * n;
        const float2 v = buf[r * n + k];
        const float2 w = __ldg(tw + k * step);
        xs[r * (n + 1) + k] = v.x * w.x - v.y * w.y;
    }
}

// Loads the inverse-DCT input X (xs, padded rows) as V_k = (X_k - i X_{n-k}) e^{i pi k / (2n)}
// into buf in bit-reversed order.
__device__ void dct3_start(float2* buf, const float* xs, int n, int logn, int R, const float2* __restrict__ tw)
{
    const int step = PD_TW / (4 * n);
    for (int e = threadIdx.x; e < R * n; e += blockDim.x) {
        const int r = e / n, k = e - r * n;
        const float a = xs[r * (n + 1) + k];
        const float b = k ? xs[r * (n + 1) + n - k] : 0.f;
        const float2 w = __ldg(tw + k * step);
        const float c = w.x, s = -w.y;  // e^{+i theta}
        buf[r * n + bitrev(k, logn)] = make_float2(a * c + b * s, a * s - b * c);
    }
}

template <int MODE>
__global__ void __launch_bounds__(PD_THREADS) k_pd_rows(PdRowArgs a)
{
    const int pair = blockIdx.y;
    if (a.ctl && (a.ctl[pair].error || (a.use_cond && !a.ctl[pair].active))) return;
    extern __shared__ __align__(16) unsigned char pd_smem[];
    const int n = a.n, logn = a.logn, R = pd_rows_per_cta(n);
    float2* buf = reinterpret_cast<float2*>(pd_smem);
    float* xs = reinterpret_cast<float*>(buf + R * n);
    const int row0 = blockIdx.x * R;
    const float* in = a.in + (size_t)pair * a.stride;
    float* out = a.out + (size_t)pair * a.stride;
    if (MODE == PD_INV) {
        // the input is a spectrum: stage it, rotate, reorder
        for (int e = threadIdx.x; e < R * n; e += blockDim.x) {
            const int r = e / n, k = e - r * n;
            xs[r * (n + 1) + k] = row0 + r < a.nrows ? in[(size_t)(row0 + r) * n + k] : 0.f;
        }
        __syncthreads();
        dct3_start(buf, xs, n, logn, R, a.tw);
    } else {
        // DCT-II input: v[i] = x[2i], v[n-1-i] = x[2i+1], at bit-reversed positions
        for (int e = threadIdx.x; e < R * n; e += blockDim.x) {
            const int r = e / n, i = e - r * n;
            const float x = row0 + r < a.nrows ? in[(size_t)(row0 + r) * n + i] : 0.f;
            const int vi = (i & 1) ? n - 1 - (i >> 1) : (i >> 1);
            buf[r * n + bitrev(vi, logn)] = make_float2(x, 0.f);
        }
    }
    __syncthreads();
    fft_rows(buf, n, logn, R, MODE == PD_INV, a.tw);
    if (MODE == PD_FWD_T) {
        dct2_finish(buf, xs, n, R, a.tw);
        __syncthreads();
        // out[k][row0 + r]: R consecutive values per k
        for (int e = threadIdx.x; e < R * n; e += blockDim.x) {
            const int k = e / R, r = e - k * R;
            if (row0 + r < a.nrows) out[(size_t)k * a.nrows + row0 + r] = xs[r * (n + 1) + k];
        }
        return;
    }
    if (MODE == PD_SOLVE_T) {
        dct2_finish(buf, xs, n, R, a.tw);
        __syncthreads();
        for (int e = threadIdx.x; e < R * n; e += blockDim.x) {
            const int r = e / n, k = e - r * n;
            const int row = row0 + r;
            float v = 0.f;
            if (row < a.nrows && (row | k)) v = xs[r * (n + 1) + k] / (__ldg(a.lam_row + row) + __ldg(a.lam_pos + k));
            xs[r * (n + 1) + k] = v;
        }
        __syncthreads();
        dct3_start(buf, xs, n, logn, R, a.tw);
        __syncthreads();
        fft_rows(buf, n, logn, R, true, a.tw);
    }
    // inverse finish: x[2i] = v[i] / n, x[2i+1] = v[n-1-i] / n (real parts)
    const float inv_n = 1.f / (float)n;
    for (int e = threadIdx.x; e < R * n; e += blockDim.x) {
        const int r = e / n, i = e - r * n;
        const int vi = (i & 1) ? n - 1 - (i >> 1) : (i >> 1);
        xs[r * (n + 1) + i] = buf[r * n + vi].x * inv_n;
    }
    __syncthreads();
    if (MODE == PD_SOLVE_T) {
        for (int e = threadIdx.x; e < R * n; e += blockDim.x) {
            const int k = e / R, r = e - k * R;
            if (row0 + r < a.nrows) out[(size_t)k * a.nrows + row0 + r] = xs[r * (n + 1) + k];
        }
    } else {
        for (int e = threadIdx.x; e < R * n; e += blockDim.x) {
            const int r = e / n, k = e - r * n;
            if (row0 + r < a.nrows) out[(size_t)(row0 + r) * n + k] = a.scale * xs[r * (n + 1) + k];
        }
    }
}

// r = div^h(v) - rho with v = m - mu phibar (pinned entries zero); pot: r = div^h(phi).
__global__ void k_pd_resid(PdArgs a, int pot)
{
    const int pair = blockIdx.z;
    if (a.ctl && (a.ctl[pair].error || (a.use_cond && !a.ctl[pair].active))) return;
    // 1-D blocks of 256 threads cover 32 x 8 nodes
    const int i = blockIdx.x * 32 + (threadIdx.x & 31), j = blockIdx.y * 8 + (threadIdx.x >> 5);
    const int nx = a.nx, ny = a.ny;
    if (i >= nx || j >= ny) return;
    const size_t o = (size_t)pair * a.stride, k = (size_t)j * nx + i;
    auto v1 = [&](size_t q, int ii) -> float {
        if (ii >= nx - 1) return 0.f;
        return pot ? a.f1[o + q] : fmaf(-a.mu, a.g1[o + q], a.m1[o + q]);
    };
    auto v2 = [&](size_t q, int jj) -> float {
        if (jj >= ny - 1) return 0.f;
        return pot ? a.f2[o + q] : fmaf(-a.mu, a.g2[o + q], a.m2[o + q]);
    };
    const float l = i > 0 ? v1(k - 1, i - 1) : 0.f;
    const float b = j > 0 ? v2(k - nx, j - 1) : 0.f;
    const float d = ((v1(k, i) - l) + (v2(k, j) - b)) * a.ih;
    a.w[o + k] = pot ? d : d - a.rho[o + k];
}

// Node-wise projection onto the unit ball of the dual norm q (p = 1: q = inf,
// p = 2: q = 2, p = inf: q = 1).
template <int NORM>
__device__ __forceinline__ void proj_dual(float v1, float v2, float& o1, float& o2)
{
    if (NORM == W1_NORM_L1) {
        o1 = fminf(fmaxf(v1, -1.f), 1.f);
        o2 = fminf(fmaxf(v2, -1.f), 1.f);
    } else if (NORM == W1_NORM_L2) {
        const float q = fmaf(v1, v1, v2 * v2);
        const float s = q > 1.f ? rsqrtf(q) : 1.f;
        o1 = v1 * s;
        o2 = v2 * s;
    } else {
        const float a = fabsf(v1), b = fabsf(v2);
        if (a + b <= 1.f) {
            o1 = v1;
            o2 = v2;
        } else {
            const float t = fabsf(a - b) >= 1.f ? fmaxf(a, b) - 1.f : 0.5f * (a + b - 1.f);
            o1 = copysignf(fmaxf(a - t, 0.f), v1);
            o2 = copysignf(fmaxf(b - t, 0.f), v2);
        }
    }
}

// m' = v + grad psi, phi' = Proj(phi + tau m'), phibar' = 2 phi' - phi; on a test
// step also the per-pair G^k (eq. pdhg_stop) and the level's stop decision.
template <int NORM, bool CHECK>
__global__ void __launch_bounds__(256) k_pd_update(PdArgs a)
{
    const int pair = blockIdx.z;
    Ctl* pc = a.ctl ? a.ctl + pair : nullptr;
    if (pc && (pc->error || (a.use_cond && !pc->active))) return;  // uniform over the pair's blocks
    // 1-D blocks of 256 threads cover 32 x 8 nodes (block_sum wants 1-D blocks)
    const int i = blockIdx.x * 32 + (threadIdx.x & 31), j = blockIdx.y * 8 + (threadIdx.x >> 5);
    const int nx = a.nx, ny = a.ny;
    float sa = 0.f, sb = 0.f, sc = 0.f;
    if (i < nx && j < ny) {
        const size_t o = (size_t)pair * a.stride, k = o + (size_t)j * nx + i;
        const float m1 = a.m1[k], m2 = a.m2[k], f1 = a.f1[k], f2 = a.f2[k];
        const float psi = a.w[k];
        float n1 = 0.f, n2 = 0.f;
        if (i < nx - 1) n1 = fmaf(-a.mu, a.g1[k], m1) + (a.w[k + 1] - psi) * a.ih;
        if (j < ny - 1) n2 = fmaf(-a.mu, a.g2[k], m2) + (a.w[k + nx] - psi) * a.ih;
        float p1, p2;
        proj_dual<NORM>(fmaf(a.tau, n1, f1), fmaf(a.tau, n2, f2), p1, p2);
        a.m1[k] = n1;
        a.m2[k] = n2;
        a.f1[k] = p1;
        a.f2[k] = p2;
        a.g1[k] = 2.f * p1 - f1;
        a.g2[k] = 2.f * p2 - f2;
        if (CHECK) {
            const float d1 = n1 - m1, d2 = n2 - m2, e1 = p1 - f1, e2 = p2 - f2;
            sa = fmaf(d1, d1, d2 * d2);
            sb = fmaf(e1, e1, e2 * e2);
            sc = fmaf(e1, d1, e2 * d2);
        }
    }
    if (!CHECK) return;
    // G^k = (|dm|^2 / mu + |dphi|^2 / tau + 2 <dphi, dm>) h^2   (eq. pdhg_stop)
    __shared__ double sh[64 * 3];
    __shared__ bool last;
    double v[3];
    ff_block_sum3(sa, sb, sc, reinterpret_cast<float*>(sh), v);
    const int nblk = gridDim.x * gridDim.y;
    const int bid = blockIdx.y * gridDim.x + blockIdx.x;
    double* pp = a.part + (size_t)pair * nblk * 3;
    const int t = threadIdx.x;
    if (t == 0) {
        pp[bid * 3 + 0] = v[0];
        pp[bid * 3 + 1] = v[1];
        pp[bid * 3 + 2] = v[2];
        __threadfence();
        last = (atomicAdd(&pc->counter, 1u) == (unsigned)nblk - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    CSum tt[3];
    for (int b = t; b < nblk; b += blockDim.x)
        for (int c = 0; c < 3; ++c) tt[c].add(((volatile double*)pp)[b * 3 + c]);
    block_csum<3>(tt, sh);
    if (t == 0) {
        const double G =
            (tt[0].value() / (double)a.mu + tt[1].value() / (double)a.tau + 2.0 * tt[2].value()) * a.h * a.h;
        pc->counter = 0;
        if (a.g_out) a.g_out[pair] = G;
        if (a.use_cond) {
            const long long it = pc->iters[a.level] + a.K;
            pc->iters[a.level] = it;
            pc->fpr[a.level] = G;
            const int conv = G < a.tol;
            pc->conv[a.level] = conv;
            const bool late = (globaltimer() - pc->t_start[a.level]) > a.budget_ns;
            if (late && !conv) pc->timeout = 1;
            if (conv || it >= a.cap || late) pc->active = 0;
        }
    }
}

size_t pd_part_doubles(int nx, int ny, int pairs)
{
    return (size_t)((nx + 31) / 32) * ((ny + 7) / 8) * pairs * 3;
}

cudaError_t pd_prepare()
{
    const int smem = (int)pd_rows_smem(PD_MAXN);
    cudaError_t e = cudaFuncSetAttribute(k_pd_rows<PD_FWD_T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pd_rows<PD_SOLVE_T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pd_rows<PD_INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return e;
}

// psi = (A A^*)^{-1} w (w holds the right-hand side on entry and psi on exit;
// dst, if not null, receives scale * psi instead)
cudaError_t launch_pd_poisson(const PdArgs& a, float* dst, float scale, cudaStream_t s)
{
    const int lx = ilog2(a.nx), ly = ilog2(a.ny);
    PdRowArgs r{};
    r.tw = a.tw;
    r.stride = a.stride;
    r.ctl = a.ctl;
    r.use_cond = a.use_cond;
    r.scale = 1.f;
    // rows (length nx) -> transposed
    r.in = a.w;
    r.out = a.t;
    r.n = a.nx;
    r.logn = lx;
    r.nrows = a.ny;
    dim3 g1((a.ny + pd_rows_per_cta(a.nx) - 1) / pd_rows_per_cta(a.nx), a.pairs);
    k_pd_rows<PD_FWD_T><<<g1, PD_THREADS, pd_rows_smem(a.nx), s>>>(r);
    // columns (length ny): forward, divide, inverse -> transposed back
    r.in = a.t;
    r.out = a.w;
    r.n = a.ny;
    r.logn = ly;
    r.nrows = a.nx;
    r.lam_row = a.lamx;
    r.lam_pos = a.lamy;
    dim3 g2((a.nx + pd_rows_per_cta(a.ny) - 1) / pd_rows_per_cta(a.ny), a.pairs);
    k_pd_rows<PD_SOLVE_T><<<g2, PD_THREADS, pd_rows_smem(a.ny), s>>>(r);
    // rows: inverse
    r.in = a.w;
    r.out = dst ? dst : a.w;
    r.n = a.nx;
    r.logn = lx;
    r.nrows = a.ny;
    r.scale = dst ? scale : 1.f;
    k_pd_rows<PD_INV><<<g1, PD_THREADS, pd_rows_smem(a.nx), s>>>(r);
    return cudaGetLastError();
}

cudaError_t launch_pd_step(int norm, bool check, const PdArgs& a, cudaStream_t s)
{
    dim3 b(256), g((a.nx + 31) / 32, (a.ny + 7) / 8, a.pairs);
    k_pd_resid<<<g, b, 0, s>>>(a, 0);
    cudaError_t e = launch_pd_poisson(a, nullptr, 1.f, s);
    if (e != cudaSuccess) return e;
    if (norm == W1_NORM_L1) {
        if (check) k_pd_update<W1_NORM_L1, true><<<g, b, 0, s>>>(a);
        else k_pd_update<W1_NORM_L1, false><<<g, b, 0, s>>>(a);
    } else if (norm == W1_NORM_L2) {
        if (check) k_pd_update<W1_NORM_L2, true><<<g, b, 0, s>>>(a);
        else k_pd_update<W1_NORM_L2, false><<<g, b, 0, s>>>(a);
    } else {
        if (check) k_pd_update<W1_NORM_LINF, true><<<g, b, 0, s>>>(a);
        else k_pd_update<W1_NORM_LINF, false><<<g, b, 0, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_pd_potential(const PdArgs& args, float* phi, cudaStream_t s)
{
    PdArgs a = args;
    a.use_cond = 0;  // after the level loop every pair is inactive; only rejected pairs are skipped
    dim3 b(256), g((a.nx + 31) / 32, (a.ny + 7) / 8, a.pairs);
    k_pd_resid<<<g, b, 0, s>>>(a, 1);
    // Appendix B: lambda = (A A^*)^{-1} A phi; the returned potential is -lambda
    // (the sign of Algorithm 1's potential, dual value -<phi, rho>_h)
    return launch_pd_poisson(a, phi, -1.f, s);
}

}  // namespace w1
