// w1_device.cuh -- device helpers shared by the kernel translation units of the
// GB300 W1 library (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "w1_internal.h"

namespace w1 {

static constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------------------
// Proximal maps (the argmin of the first line of eq. primaldual)
// ---------------------------------------------------------------------------

__device__ __forceinline__ float soft(float v, float mu)
{
    // sign(v) max(|v| - mu, 0), written as v minus its clamp to [-mu, mu]
    return v - fminf(fmaxf(v, -mu), mu);
}

template <int NORM>
__device__ __forceinline__ void prox(float v1, float v2, float mu, float& o1, float& o2)
{
    if (NORM == W1_NORM_L1) {
        o1 = soft(v1, mu);
        o2 = soft(v2, mu);
    } else if (NORM == W1_NORM_LINF) {
        // v - mu * Proj_{l1 ball}(v / mu) (Moreau): zero inside the ball; else the
        // larger component loses mu, or both magnitudes meet at (|v1| + |v2| - mu) / 2
        const float a = fabsf(v1), b = fabsf(v2);
        if (a + b <= mu) {
            o1 = 0.f;
            o2 = 0.f;
        } else if (a - b >= mu) {
            o1 = copysignf(a - mu, v1);
            o2 = v2;
        } else if (b - a >= mu) {
            o1 = v1;
            o2 = copysignf(b - mu, v2);
        } else {
            const float c = 0.5f * (a + b - mu);
            o1 = copysignf(c, v1);
            o2 = copysignf(c, v2);
        }
    } else {
        // v max(0, 1 - mu / |v|); rsqrt(0) = inf gives 0
        const float s = fmaxf(1.f - mu * rsqrtf(fmaf(v1, v1, v2 * v2)), 0.f);
        o1 = v1 * s;
        o2 = v2 * s;
    }
}

// Packed FP32 (two lanes per instruction, sm_100+): the same IEEE round-to-
// nearest operations as the scalar forms, two at a time; a - b is written as
// a + (-b), which rounds identically.
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }
__device__ __forceinline__ float2 splat2(float a) { return make_float2(a, a); }

// prox of two nodes at once, each given as (component 1 of nodes a, b) and
// (component 2 of nodes a, b); p = infinity falls back to the scalar form
template <int NORM>
__device__ __forceinline__ void prox_pair(float2 v1, float2 v2, float mu, float2& o1, float2& o2)
{
    if (NORM == W1_NORM_L1) {
        const float2 c1 = make_float2(fminf(fmaxf(v1.x, -mu), mu), fminf(fmaxf(v1.y, -mu), mu));
        const float2 c2 = make_float2(fminf(fmaxf(v2.x, -mu), mu), fminf(fmaxf(v2.y, -mu), mu));
        o1 = sub2(v1, c1);
        o2 = sub2(v2, c2);
    } else if (NORM == W1_NORM_L2) {
        const float2 q = __ffma2_rn(v1, v1, __fmul2_rn(v2, v2));
        const float2 r = make_float2(rsqrtf(q.x), rsqrtf(q.y));
        const float2 t = __ffma2_rn(splat2(-mu), r, splat2(1.f));
        const float2 s = make_float2(fmaxf(t.x, 0.f), fmaxf(t.y, 0.f));
        o1 = __fmul2_rn(v1, s);
        o2 = __fmul2_rn(v2, s);
    } else {
        prox<NORM>(v1.x, v2.x, mu, o1.x, o2.x);
        prox<NORM>(v1.y, v2.y, mu, o1.y, o2.y);
    }
}

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Distributed shared memory through 32-bit shared::cluster addresses (cheaper
// in registers than generic 64-bit pointers).
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint32_t dsmem_map(uint32_t addr, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
__device__ __forceinline__ float dsmem_ld(uint32_t addr)
{
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ float4 dsmem_ld4(uint32_t addr)
{
    float4 v;
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(addr)
                 : "memory");
    return v;
}
__device__ __forceinline__ void dsmem_st_f64(uint32_t addr, double v)
{
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}
__device__ __forceinline__ void dsmem_st_u32(uint32_t addr, unsigned v)
{
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ double dsmem_ld_f64(uint32_t addr)
{
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(addr) : "memory");
    return v;
}

// Neighbour-to-neighbour exchange inside a cluster: a CTA pushes a row into
// the neighbour's shared memory with st.async, whose bytes complete a
// transaction count on an mbarrier of the receiving CTA; the receiver arms the
// barrier with the bytes it expects and waits on its phase parity.
__device__ __forceinline__ void mbar_init(uint32_t bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// Ends the barrier object, so that its memory can hold a new one (a persistent
// launch initialises the halo barriers again for every level it solves).
__device__ __forceinline__ void mbar_inval(uint32_t bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect(uint32_t bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
// try_wait suspends the thread until the phase completes or about
// MBAR_SUSPEND_NS have passed, so a waiting warp does not take issue slots
// from the warps that still compute by polling.
static constexpr unsigned MBAR_SUSPEND_NS = 20000;
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, unsigned parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "n"(MBAR_SUSPEND_NS)
        : "memory");
    return ok != 0;
}
// Waits for the phase with the given parity to complete; false after about
// limit_ns of wall-clock time (the caller records the failure and carries on).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, unsigned parity, unsigned long long limit_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (globaltimer() - t0 > limit_ns) return false;
    }
}
// 16 bytes into a neighbour CTA's shared memory (both addresses from mapa).
__device__ __forceinline__ void st_async4(uint32_t addr, float4 v, uint32_t bar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(
                     addr),
                 "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(bar)
                 : "memory");
}

// Tensor memory (TMEM) as per-thread storage beside the registers: one warp
// allocates columns for the CTA, every warp reads and writes the 32 lanes of
// its quarter (lanes 32 (warp % 4) .. + 31), one 32-bit cell per lane and
// column; addresses are (lane << 16) | column relative to the allocation.
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Four consecutive columns of the thread's lane; the wait for the load is in
// the same asm statement, so no code can touch the registers before they land.
__device__ __forceinline__ float4 tmem_ld4(uint32_t taddr)
{
    uint32_t a, b, c, d;
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(a), "=r"(b), "=r"(c), "=r"(d)
        : "r"(taddr)
        : "memory");
    return make_float4(__uint_as_float(a), __uint_as_float(b), __uint_as_float(c), __uint_as_float(d));
}
__device__ __forceinline__ void tmem_st4(uint32_t taddr, float4 v)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr),
                 "r"(__float_as_uint(v.x)), "r"(__float_as_uint(v.y)), "r"(__float_as_uint(v.z)),
                 "r"(__float_as_uint(v.w))
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
// The same with a compile-time column offset folded into the address operand.
template <int OFF>
__device__ __forceinline__ float4 tmem_ld4_at(uint32_t taddr)
{
    uint32_t a, b, c, d;
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4+%5];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(a), "=r"(b), "=r"(c), "=r"(d)
        : "r"(taddr), "n"(OFF)
        : "memory");
    return make_float4(__uint_as_float(a), __uint_as_float(b), __uint_as_float(c), __uint_as_float(d));
}
template <int OFF>
__device__ __forceinline__ void tmem_st4_at(uint32_t taddr, float4 v)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0+%1], {%2, %3, %4, %5};" ::"r"(taddr), "n"(OFF),
                 "r"(__float_as_uint(v.x)), "r"(__float_as_uint(v.y)), "r"(__float_as_uint(v.z)),
                 "r"(__float_as_uint(v.w))
                 : "memory");
}

// Two and four loads of four columns each behind one wait: the loads are in
// flight together, and no code can touch the registers before all have landed.
template <int O0, int O1>
__device__ __forceinline__ void tmem_ld4x2_at(uint32_t taddr, float4& a, float4& b)
{
    uint32_t r[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%8+%9];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%4, %5, %6, %7}, [%8+%10];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "r"(taddr), "n"(O0), "n"(O1)
        : "memory");
    a = make_float4(__uint_as_float(r[0]), __uint_as_float(r[1]), __uint_as_float(r[2]), __uint_as_float(r[3]));
    b = make_float4(__uint_as_float(r[4]), __uint_as_float(r[5]), __uint_as_float(r[6]), __uint_as_float(r[7]));
}
template <int O0, int O1, int O2, int O3>
__device__ __forceinline__ void tmem_ld4x4_at(uint32_t taddr, float4& a, float4& b, float4& c, float4& d)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%16+%17];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%4, %5, %6, %7}, [%16+%18];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%8, %9, %10, %11}, [%16+%19];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%12, %13, %14, %15}, [%16+%20];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr), "n"(O0), "n"(O1), "n"(O2), "n"(O3)
        : "memory");
    a = make_float4(__uint_as_float(r[0]), __uint_as_float(r[1]), __uint_as_float(r[2]), __uint_as_float(r[3]));
    b = make_float4(__uint_as_float(r[4]), __uint_as_float(r[5]), __uint_as_float(r[6]), __uint_as_float(r[7]));
    c = make_float4(__uint_as_float(r[8]), __uint_as_float(r[9]), __uint_as_float(r[10]), __uint_as_float(r[11]));
    d = make_float4(__uint_as_float(r[12]), __uint_as_float(r[13]), __uint_as_float(r[14]), __uint_as_float(r[15]));
}

// Calls f(std::integral_constant<int, r>{}) for r = 0 .. N - 1 (a loop whose
// index is a compile-time constant in the body).
template <int N, class F>
__device__ __forceinline__ void static_for(F&& f)
{
    if constexpr (N > 0) {
        static_for<N - 1>(f);
        f(std::integral_constant<int, N - 1>{});
    }
}

// Split cluster barrier (release on arrive, acquire on wait).
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

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

// ---------------------------------------------------------------------------
// Compensated sums
// ---------------------------------------------------------------------------
//
// Knuth's TwoSum gives s = fl(a + b) and the exact rounding error e, so that
// s + e == a + b exactly.  The explicitly rounded intrinsics keep the compiler
// from contracting or reordering the steps.  A compensated sum (Neumaier's
// scheme, with the exact error term of every addition) carries the
// running value as the unevaluated pair s + c: its error is about one rounding
// of the result plus n u^2 sum|x_i|, instead of about n u sum|x_i| for a plain
// left-to-right sum (u the unit roundoff).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// s = fl(a + b) and its exact rounding error e from Dekker's Fast2Sum on the operands ordered by
// magnitude (Neumaier's comparison): e = (big - s) + small is exact when
// |big| >= |small|.  Three FP64 additions and a comparison instead of six
// additions; the selects run on the integer pipe.  GB300 issues FP64 at a
// small fraction of its FP32 rate, so the compensated sums use this form.
__device__ __forceinline__ void two_sum_ordered(double a, double b, double& s, double& e)
{
    s = __dadd_rn(a, b);
    const bool ge = fabs(a) >= fabs(b);
    const double big = ge ? a : b, small = ge ? b : a;
    e = __dadd_rn(__dsub_rn(big, s), small);
}

struct CSum {
    double s = 0.0, c = 0.0;
    __device__ __forceinline__ void add(double x)
    {
        double t, e;
        two_sum_ordered(s, x, t, e);
        s = t;
        c = __dadd_rn(c, e);
    }
    // adds another compensated sum
    __device__ __forceinline__ void add(const CSum& o)
    {
        double t, e;
        two_sum_ordered(s, o.s, t, e);
        s = t;
        c = __dadd_rn(c, __dadd_rn(o.c, e));
    }
    __device__ __forceinline__ double value() const { return __dadd_rn(s, c); }
};

// Compensated sums of N values over the block, in a fixed order (lanes by
// shuffles, then the warps' sums in warp 0); result valid in thread 0.
// sh: 64*N doubles.
template <int N>
__device__ void block_csum(CSum (&v)[N], double* sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int c = 0; c < N; ++c) {
            CSum r;
            r.s = __shfl_xor_sync(FULL, v[c].s, o);
            r.c = __shfl_xor_sync(FULL, v[c].c, o);
            v[c].add(r);
        }
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < N; ++c) {
            sh[(warp * N + c) * 2] = v[c].s;
            sh[(warp * N + c) * 2 + 1] = v[c].c;
        }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int c = 0; c < N; ++c) {
            v[c].s = (lane < nw) ? sh[(lane * N + c) * 2] : 0.0;
            v[c].c = (lane < nw) ? sh[(lane * N + c) * 2 + 1] : 0.0;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int c = 0; c < N; ++c) {
                CSum r;
                r.s = __shfl_xor_sync(FULL, v[c].s, o);
                r.c = __shfl_xor_sync(FULL, v[c].c, o);
                v[c].add(r);
            }
    }
    __syncthreads();
}

// The same sums through shared memory, for blocks whose lanes would otherwise
// spend most of a shuffle tree adding zeros in FP64: every thread stores its N
// sums, then each level adds the upper half of every sum's column into its
// lower half, the N columns sharing the level's threads.  A level of width w
// costs N w additions in total instead of N per lane.  Fixed order; result
// valid in thread 0.  sh: 2 N blockDim.x doubles; blockDim.x a power of two.
template <int N>
__device__ void block_csum_sh(CSum (&v)[N], double* sh)
{
    const int T = blockDim.x, tid = threadIdx.x;
    double* S = sh;
    double* C = sh + N * T;
    __syncthreads();
#pragma unroll
    for (int c = 0; c < N; ++c) {
        S[c * T + tid] = v[c].s;
        C[c * T + tid] = v[c].c;
    }
    __syncthreads();
    for (int w = T / 2; w >= 1; w >>= 1) {
        for (int idx = tid; idx < N * w; idx += T) {
            const int c = idx / w, k = c * T + (idx - c * w);
            CSum a, b;
            a.s = S[k];
            a.c = C[k];
            b.s = S[k + w];
            b.c = C[k + w];
            a.add(b);
            S[k] = a.s;
            C[k] = a.c;
        }
        __syncthreads();
    }
    if (tid == 0)
#pragma unroll
        for (int c = 0; c < N; ++c) {
            v[c].s = S[c * T];
            v[c].c = C[c * T];
        }
    __syncthreads();  // sh free for the caller again
}

// Block sums of three per-thread FP32 values (the terms of the stop test),
// compensated in float pairs: every addition is a TwoSum whose error goes into
// the pair's low part, first across the lanes of each warp, then across the
// warps' pairs in warp 0.  GB300's FP64 rate is a small fraction of its FP32
// rate, so the block-wide tree stays in FP32 pairs (about 48 significant bits);
// thread 0 gets each sum as FP64 hi + lo.  sh: at least 32 * 6 floats.
__device__ __forceinline__ void ff_warp_add(float& hi, float& lo, int o)
{
    const float h2 = __shfl_xor_sync(FULL, hi, o), l2 = __shfl_xor_sync(FULL, lo, o);
    float s, e;
    two_sum(hi, h2, s, e);
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(l2, e));
}
// one value at a time (few live registers: this runs inside the level kernels)
__device__ __forceinline__ void ff_warp_sum(float x, float& hi, float& lo)
{
    hi = x;
    lo = 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ff_warp_add(hi, lo, o);
}
static __device__ __noinline__ void ff_block_sum3(float a, float b, float c, float* sh, double (&out)[3])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    float hi, lo;
    __syncthreads();
    ff_warp_sum(a, hi, lo);
    if (lane == 0) {
        sh[warp * 6] = hi;
        sh[warp * 6 + 1] = lo;
    }
    ff_warp_sum(b, hi, lo);
    if (lane == 0) {
        sh[warp * 6 + 2] = hi;
        sh[warp * 6 + 3] = lo;
    }
    ff_warp_sum(c, hi, lo);
    if (lane == 0) {
        sh[warp * 6 + 4] = hi;
        sh[warp * 6 + 5] = lo;
    }
    __syncthreads();
    if (warp == 0) {
        for (int k = 0; k < 3; ++k) {
            hi = lane < nw ? sh[lane * 6 + 2 * k] : 0.f;
            lo = lane < nw ? sh[lane * 6 + 2 * k + 1] : 0.f;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) ff_warp_add(hi, lo, o);
            out[k] = (double)hi + (double)lo;
        }
    }
    __syncthreads();
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

}  // namespace w1
