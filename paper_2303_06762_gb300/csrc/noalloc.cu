// hdg_restrict_noalloc: the restriction of the lowest-order transfer with its
// coarse-cell scratch in a fixed array compiled into the library, for callers
// that cannot allocate device memory.  The paper has no counterpart; this is
// an interface convenience only.
//
// The scratch is a file-scope __device__ array.  Host code cannot use the
// array's name as a device address, so the first call on each device (with
// that device current) asks the runtime for the array's device address with
// cudaGetSymbolAddress and caches it; later calls on that device reuse it.
// Nothing here calls cudaMalloc, cudaFree or any allocating routine.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "hdg_internal.h"

namespace {

constexpr int kMaxDevices = 64;
constexpr int kPerCell = 18;      // 12 (H^T r_T) + 6 (W^T z) doubles per coarse cell

static __device__ __align__(256) double g_restrict_scratch[(size_t)HDG_NOALLOC_MAX_COARSE_CELLS * kPerCell];

std::mutex g_mutex;
double *g_addr[kMaxDevices] = {nullptr};

// the body of hdg_restrict_noalloc; may throw only from the host string and lock operations
hdg_status restrict_noalloc_impl(hdg_ctx *ctx, int level, const double *rf, double *rc, hdg_stream_t stream) {
    if (!ctx->condensed) {
        ctx->err = "hdg_restrict_noalloc: operator used before hdg_condense";
        return HDG_ERR_STATE;
    }
    if (level < 1 || level >= ctx->n_levels || !rf || !rc) {
        ctx->err = "hdg_restrict_noalloc: level out of range 1..n_levels-1 or null vector";
        return HDG_ERR_INVALID_ARG;
    }
    const hdg::DevLevel &F = ctx->L[level];
    if (F.nc_coarse > (int64_t)HDG_NOALLOC_MAX_COARSE_CELLS) {
        ctx->err = "hdg_restrict_noalloc: the coarse level has " + std::to_string(F.nc_coarse) +
                   " cells, more than the fixed scratch holds (" +
                   std::to_string(HDG_NOALLOC_MAX_COARSE_CELLS) + "); use hdg_restrict";
        return HDG_ERR_INVALID_ARG;
    }
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        ctx->err = std::string("hdg_restrict_noalloc: cudaGetDevice: ") + cudaGetErrorString(e);
        return HDG_ERR_CUDA;
    }
    if (dev != ctx->device) {
        ctx->err = "hdg_restrict_noalloc: the current device is not the context's device";
        return HDG_ERR_INVALID_ARG;
    }
    double *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_restrict_scratch);
            if (e != cudaSuccess || !p) {
                ctx->err = std::string("hdg_restrict_noalloc: cudaGetSymbolAddress: ") +
                           cudaGetErrorString(e);
                return HDG_ERR_CUDA;
            }
            g_addr[dev] = static_cast<double *>(p);
        }
        scratch = g_addr[dev];
    }
    // the two temporaries are written in full before they are read: no clearing needed
    double *t1 = scratch;
    double *t2 = scratch + (size_t)12 * F.nc_coarse;
    e = hdg::launch_restrict<double>(F, ctx->L[level - 1], F.tr_W.p, F.tr_H.p, rf, t1, t2, rc,
                                     (cudaStream_t)stream);
    if (e != cudaSuccess) {
        ctx->err = std::string("hdg_restrict_noalloc: ") + cudaGetErrorString(e);
        return HDG_ERR_CUDA;
    }
    return HDG_OK;
}

} // namespace

extern "C" hdg_status hdg_restrict_noalloc(hdg_ctx *ctx, int level, const double *rf, double *rc,
                                           hdg_stream_t stream) {
    if (!ctx) return HDG_ERR_INVALID_ARG;
    // no exception may cross the C ABI (a failed string or lock operation is reported instead)
    try {
        return restrict_noalloc_impl(ctx, level, rf, rc, stream);
    } catch (...) {
        try {
            ctx->err = "hdg_restrict_noalloc: host-side exception";
        } catch (...) {
        }
        return HDG_ERR_INVALID_ARG;
    }
}
