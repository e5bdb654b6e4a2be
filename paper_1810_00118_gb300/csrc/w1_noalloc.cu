// w1_noalloc.cu -- statistics of a state without any device allocation.
//
// w1_state_stats allocates its scratch (FP64 residual masses for the route
// bound, per-block partial sums, a control block) with cudaMalloc on every
// call.  Some callers cannot do that: code that must not trigger the implicit
// device synchronisation of cudaMalloc/cudaFree in a latency-critical loop,
// hosts whose framework owns every byte of device memory through its own pool,
// and services that run in a fixed, preallocated footprint.  This file gives
// them w1_state_stats_noalloc: the same kernels, with the scratch in a
// file-scope static device array that every GPU loading this library holds
// until the process exits.  The call copies the statistics to the host and
// synchronises the stream before it returns.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>

#include "w1_internal.h"

using namespace w1;

namespace {

constexpr size_t kAlign = 256;
constexpr size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Layout of the static scratch: control block | partial sums | 2 * n FP64 masses.
constexpr size_t kCtlBytes = align_up(sizeof(Ctl));
constexpr size_t kPartBytes = align_up(304 * 5 * sizeof(double));
// the final statistics' partial sums of one pair must fit their reserve
static_assert((size_t)FIN_BLOCKS_PER_PAIR * FIN_PART_PER_BLOCK * sizeof(double) <= kPartBytes,
              "partial-sum reserve smaller than final_part_doubles(1)");
constexpr size_t kQBytes = 2 * (size_t)W1_NOALLOC_MAX_NODES * sizeof(double);
constexpr size_t kScratchBytes = kCtlBytes + kPartBytes + kQBytes;

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

thread_local std::string g_na_err;
std::mutex g_na_mu;
void* g_na_base[64] = {};

w1_status na_fail(w1_status s, const std::string& m)
{
    g_na_err = m;
    return s;
}

}  // namespace

// The last error of this entry point (kept apart from w1_last_error so that
// neither path overwrites the other's message).
extern "C" const char* w1_noalloc_last_error(void) { return g_na_err.c_str(); }

extern "C" w1_status w1_state_stats_noalloc(int nx, int ny, double h, int norm, const float* rho, const float* m1,
                                            const float* m2, const float* phi, void* stream, w1_stats* out)
{
    if (nx < 1 || ny < 1 || !(h > 0.0) || !rho || !m1 || !m2 || !phi || !out)
        return na_fail(W1_ERR_INVALID_ARG, "bad arguments to w1_state_stats_noalloc");
    if (norm != W1_NORM_L1 && norm != W1_NORM_L2 && norm != W1_NORM_LINF) return na_fail(W1_ERR_INVALID_ARG, "norm must be 1, 2 or 3");
    if ((long long)nx * (long long)ny > (long long)W1_NOALLOC_MAX_NODES)
        return na_fail(W1_ERR_INVALID_ARG, "grid has more than W1_NOALLOC_MAX_NODES (262144) nodes");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(W1_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= 64) return na_fail(W1_ERR_UNSUPPORTED, "device index above 63");
    void* base = nullptr;
    {
        // Set-up, once per device with that device current: the array's name is
        // only a host-side stand-in, so fetch its device address.
        std::lock_guard<std::mutex> lk(g_na_mu);
        if (!g_na_base[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return na_fail(W1_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            }
            g_na_base[dev] = p;
        }
        base = g_na_base[dev];
    }
    unsigned char* b = static_cast<unsigned char*>(base);
    Ctl* ctl = reinterpret_cast<Ctl*>(b);
    double* part = reinterpret_cast<double*>(b + kCtlBytes);
    double* q = reinterpret_cast<double*>(b + kCtlBytes + kPartBytes);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // The array keeps the previous call's contents: the control block must start at zero.
    e = cudaMemsetAsync(ctl, 0, sizeof(Ctl), s);
    if (e == cudaSuccess) e = launch_final(norm, m1, m2, phi, rho, nx, ny, h, q, part, ctl, 1, s);
    Ctl c;
    std::memset(&c, 0, sizeof(c));
    if (e == cudaSuccess) e = cudaMemcpyAsync(&c, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return na_fail(W1_ERR_CUDA, std::string("w1_state_stats_noalloc: ") + cudaGetErrorString(e));
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
