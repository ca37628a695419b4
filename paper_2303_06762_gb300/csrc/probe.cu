// Measurement utility: the FP64 fused multiply-add rate of this GPU, the
// arithmetic ceiling of the FP64 kernels (outer operator apply, Krylov passes).
// The paper has no counterpart; it supplies the FP64 denominator of a roofline.
//
// Every thread runs CHAINS independent FMA chains a <- a*b + c for `iters`
// iterations (b, c are runtime values, so nothing folds), enough chains to
// cover the FMA latency; the grid fills every SM several times over.
#include <cuda_runtime.h>

#include "hdg_internal.h"

namespace {

constexpr int CHAINS = 8;
constexpr int THREADS = 256;

__global__ void __launch_bounds__(THREADS) fp64_fma_kernel(long long iters, double b, double c, double *out) {
    double a[CHAINS];
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) a[i] = (double)(threadIdx.x + i) * 1e-3;
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < CHAINS; ++i) a[i] = fma(a[i], b, c);
    }
    double s = 0;
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) s += a[i];
    if (s == 1234.5678) out[0] = -s;   // keeps every thread's chains live; never true for these inputs
    if (threadIdx.x == 0 && blockIdx.x == 0) out[0] = s;
}

} // namespace

extern "C" int64_t hdg_fp64_fma_probe(int blocks_per_sm, int64_t iters, double *out, hdg_stream_t stream) {
    if (blocks_per_sm < 1 || blocks_per_sm > 64 || iters < 1 || !out) return -1;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
    const int blocks = sms * blocks_per_sm;
    hdg::note_launches(1);
    fp64_fma_kernel<<<blocks, THREADS, 0, (cudaStream_t)stream>>>((long long)iters, 0.999999, 1e-7, out);
    if (cudaGetLastError() != cudaSuccess) return -1;
    return (int64_t)2 * CHAINS * THREADS * blocks * iters;
}
