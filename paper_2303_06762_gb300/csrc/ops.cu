// Hot-path kernels of the hp-multigrid preconditioned FGMRES (FP64 / FP32).
//
// * apply: y = Σ_K E_Kᵀ A_K E_K x (eqs. stOptForm, stALform), computed per
//   skeleton unknown: the row of every interior facet is the sum of the rows
//   of the two adjacent cells' condensed matrices against the gathered facet
//   values of those cells.  No atomics; every output written once.
// * gs_colour: one phase of multicolour block Gauss–Seidel over vertex
//   patches (eq. bjac with GS, Section 5): every patch of the colour forms its
//   residual rows from the cells of its star, multiplies by the stored patch
//   inverse and updates its unknowns.  Patches of one colour share no cell, so
//   the phase equals the sequential sweep over those patches.  Variants: the
//   order-k FP32 phase with its matrices staged by cp.async.bulk
//   (gs_tma_kernel), the lowest-order phase with lane groups per patch
//   (gs0_kernel) and, on small levels, through a gather table (gs0t_kernel).
// * hp transfers (Section 3.5): Π_k^0 takes the m = 0 normal and tangential
//   coefficient of every facet; Π_0^k adds them back.
// * CR transfers (eqs. avgOpt, div-transfer, harmonic-ex): prolongation
//   = averaging of the coarse Π^CR values at fine boundary-facet midpoints
//   followed by the harmonic extension H = −A_TT⁻¹A_TB inside every coarse
//   cell; restriction = its exact transpose.
// * Krylov: fused classical Gram–Schmidt passes (dots, update+dots,
//   update+norm) with deterministic two-stage reductions, Givens rotations
//   and the triangular solve on the device.
// * Uzawa (eq. stOpEq-ALU): load F + Dᵀp and the cell-wise pressure update.
//
// Element matrices are stored by facet row blocks and patch inverses as their
// transposes, so that consecutive threads (consecutive rows) touch consecutive
// addresses.  The order-k apply and sweep also read 16-bit copies (bfloat16 or
// binary16) whose rows carry a power-of-two scale; products accumulate in FP32.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <type_traits>

#include "hdg3d_internal.h"

namespace hdg {

static std::atomic<unsigned long long> g_launches{0};
thread_local unsigned long long t_launches = 0;   // launches enqueued by this host thread
void note_launches(long long n) {
    g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed);
    t_launches += (unsigned long long)n;
}
unsigned long long launch_count() { return g_launches.load(std::memory_order_relaxed); }
unsigned long long thread_launch_count() { return t_launches; }

namespace {

constexpr int KRYLOV_BLOCKS = 456;    // 3 x 152 SMs
constexpr int KRYLOV_THREADS = 256;
constexpr int MAXV = 65;              // restart <= 64: up to 65 basis vectors

unsigned blocks_for(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// value of a stored matrix entry in the arithmetic type T
template <class T>
__device__ __forceinline__ T ld_entry(const T *p) { return *p; }
__device__ __forceinline__ float ld_entry(const __half *p) { return __half2float(*p); }
__device__ __forceinline__ float ld_entry(const __nv_bfloat16 *p) { return __bfloat162float(*p); }

// S = storage type of A (T, or a 16-bit type with per-row scales As[c*NLOC + row])
template <class T, int DPF, class S = T>
__global__ void __launch_bounds__(256)
apply_kernel(int64_t n_int, const int *__restrict__ facet_adj, const int *__restrict__ cell_int,
             const S *__restrict__ A, const float *__restrict__ As, const T *__restrict__ x,
             const T *__restrict__ g, T *__restrict__ y) {
    constexpr int NLOC = 3 * DPF;
    constexpr bool scaled = !std::is_same<S, T>::value;
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n_int * DPF) return;
    int64_t i = idx / DPF;
    int d = (int)(idx - i * DPF);
    T acc = 0;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        int adj = facet_adj[2 * i + q];
        if (adj < 0) continue;
        int c = adj >> 2, lf = adj & 3;
        const S *Ac = A + (size_t)c * NLOC * NLOC + lf * NLOC * DPF + d;
        T part = 0;
#pragma unroll
        for (int f2 = 0; f2 < 3; ++f2) {
            int j = cell_int[3 * c + f2];
            if (j < 0) continue;
            const T *xs = x + (size_t)j * DPF;
            if constexpr (scaled) {
#pragma unroll
                for (int d2 = 0; d2 < DPF; ++d2) part += ld_entry(Ac + (f2 * DPF + d2) * DPF) * xs[d2];
            } else {
#pragma unroll
                for (int d2 = 0; d2 < DPF; ++d2) acc += Ac[(f2 * DPF + d2) * DPF] * xs[d2];
            }
        }
        if constexpr (scaled) acc += As[(size_t)c * NLOC + lf * DPF + d] * part;
    }
    y[idx] = g ? g[idx] - acc : acc;
}

// S = storage type of A and Pinv (T, or a 16-bit type with per-row scales As[c*NLOC + row]
// and Ps[p*np_max + row] of the element matrices and patch inverses).
// EXT: the closed-form update u_P = A_PP^-1 (g_P - A_PE u_E) (E = each star cell's facet
// opposite the patch vertex, patch_cext), which equals the correction form
// u_P + A_PP^-1 (g - A u)_P because Pinv inverts the assembled A_PP; it reads the DPF x DPF
// coupling blocks instead of whole facet row blocks, and the unknowns on E only.  With swQ
// (the FP32 sweep) the AL term is split off as in gs_tma_kernel: A_PP^-1 (g_P - A0_PE u_E) - Q z.
template <class T, int DPF, class S = T, bool EXT = false>
__global__ void gs_kernel(int p0, int p1, int pf_max, int pc_max, int np_max,
                          const int *__restrict__ patch_nf, const int *__restrict__ patch_facets,
                          const int *__restrict__ patch_nc, const int *__restrict__ patch_cells,
                          const int *__restrict__ slot_src, const int *__restrict__ cell_int,
                          const int *__restrict__ patch_cext, const float *__restrict__ swQ,
                          const float *__restrict__ swA00, const double *__restrict__ cell_d,
                          const S *__restrict__ A, const float *__restrict__ As,
                          const S *__restrict__ Pinv, const float *__restrict__ Ps,
                          const T *__restrict__ g, T *__restrict__ u) {
    constexpr int NLOC = 3 * DPF;
    constexpr int NX = EXT ? DPF : NLOC;        // gathered unknowns per star cell
    constexpr bool scaled = !std::is_same<S, T>::value;
    extern __shared__ __align__(16) unsigned char smraw[];
    T *xs = reinterpret_cast<T *>(smraw);     // pc_max * NX
    T *r = xs + pc_max * NX;                   // np_max
    T *zs = r + np_max;                        // pc_max outside fluxes (split form)
    const int p = p0 + blockIdx.x;
    if (p >= p1) return;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int nf = patch_nf[p], ncell = patch_nc[p], np = nf * DPF;
    const bool split = EXT && swQ;
    for (int t = tid; t < ncell * NX; t += nt) {
        const int si = t / NX, l = t % NX;
        const int c = patch_cells[(size_t)p * pc_max + si];
        const int f = EXT ? patch_cext[(size_t)p * pc_max + si] : l / DPF;
        const int j = cell_int[3 * c + f];
        const T x = j >= 0 ? u[(size_t)j * DPF + l % DPF] : T(0);
        xs[t] = x;
        if (split && l == 0) zs[si] = (T)cell_d[3 * (size_t)c + f] * x;
    }
    __syncthreads();
    for (int t = tid; t < np; t += nt) {
        int js = t / DPF, d = t % DPF;
        int F = patch_facets[(size_t)p * pf_max + js];
        T acc = g[(size_t)F * DPF + d];
        for (int q = 0; q < 2; ++q) {
            int src = slot_src[((size_t)p * pf_max + js) * 2 + q];
            int si = src >> 2, lf = src & 3;
            int c = patch_cells[(size_t)p * pc_max + si];
            const int col0 = EXT ? patch_cext[(size_t)p * pc_max + si] * DPF : 0;
            const S *Ac = A + (size_t)c * NLOC * NLOC + lf * NLOC * DPF + col0 * DPF + d;
            const T *xc = xs + si * NX;
            if constexpr (scaled) {
                T part = 0;
#pragma unroll
                for (int col = 0; col < NX; ++col) part += ld_entry(Ac + col * DPF) * xc[col];
                acc -= As[(size_t)c * NLOC + lf * DPF + d] * part;
            } else {
                const T a00 = (split && d == 0) ? (T)swA00[((size_t)p * pf_max + js) * 2 + q] : Ac[0];
                acc -= a00 * xc[0];
#pragma unroll
                for (int col = 1; col < NX; ++col) acc -= Ac[col * DPF] * xc[col];
            }
        }
        r[t] = acc;
    }
    __syncthreads();
    const S *Pi = Pinv + (size_t)p * np_max * np_max;
    for (int t = tid; t < np; t += nt) {
        // four partial sums keep several independent loads in flight per thread
        T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        int j = 0;
#pragma unroll 2
        for (; j + 4 <= np; j += 4) {
            a0 += ld_entry(Pi + (size_t)(j + 0) * np_max + t) * r[j + 0];
            a1 += ld_entry(Pi + (size_t)(j + 1) * np_max + t) * r[j + 1];
            a2 += ld_entry(Pi + (size_t)(j + 2) * np_max + t) * r[j + 2];
            a3 += ld_entry(Pi + (size_t)(j + 3) * np_max + t) * r[j + 3];
        }
        for (; j < np; ++j) a0 += ld_entry(Pi + (size_t)j * np_max + t) * r[j];
        if (split)
            for (int si = 0; si < ncell; ++si) a2 -= (T)swQ[((size_t)p * pc_max + si) * np_max + t] * zs[si];
        T du = (a0 + a1) + (a2 + a3);
        if constexpr (scaled) du *= Ps[(size_t)p * np_max + t];
        int F = patch_facets[(size_t)p * pf_max + t / DPF];
        if constexpr (EXT) u[(size_t)F * DPF + t % DPF] = du;
        else u[(size_t)F * DPF + t % DPF] += du;
    }
}

// 16-bit row-scaled copies of the order-k element matrices: one thread per stored row
// (cell c, row p = lf*DPF + d); s = 2^e with max_q |A_pq| = m 2^e, m in [1/2, 1).
template <class S>
__device__ __forceinline__ S to_storage(double v);
template <>
__device__ __forceinline__ __half to_storage<__half>(double v) { return __double2half(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 to_storage<__nv_bfloat16>(double v) { return __double2bfloat16(v); }

__device__ __forceinline__ double pow2_scale(double m) {
    if (!(m > 0.0) || !isfinite(m)) return 1.0;
    int e;
    frexp(m, &e);
    return ldexp(1.0, e);
}

template <class S, int DPF>
__global__ void round_element_rows_kernel(int64_t nc, const double *__restrict__ A, S *__restrict__ Ah,
                                          float *__restrict__ As) {
    constexpr int NLOC = 3 * DPF;
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= nc * NLOC) return;
    const int64_t c = idx / NLOC;
    const int row = (int)(idx - c * NLOC), lf = row / DPF, d = row % DPF;
    const size_t base = (size_t)c * NLOC * NLOC + (size_t)lf * NLOC * DPF + d;
    double m = 0.0;
    for (int q = 0; q < NLOC; ++q) m = fmax(m, fabs(A[base + (size_t)q * DPF]));
    const double sc = pow2_scale(m);
    for (int q = 0; q < NLOC; ++q) Ah[base + (size_t)q * DPF] = to_storage<S>(A[base + (size_t)q * DPF] / sc);
    As[idx] = (float)sc;
}

// the same for the patch inverses, stored transposed (row i of the inverse at
// Pinv[j*np_max + i]); rows and columns beyond the patch's own size become zero
template <class S>
__global__ void round_patch_rows_kernel(int n_patches, int np_max, int dpf, const int *__restrict__ patch_nf,
                                        const double *__restrict__ P, S *__restrict__ Ph,
                                        float *__restrict__ Ps) {
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n_patches * np_max) return;
    const int64_t pt = idx / np_max;
    const int i = (int)(idx - pt * np_max);
    const int np = patch_nf[pt] * dpf;
    const size_t base = (size_t)pt * np_max * np_max + i;
    double m = 0.0;
    if (i < np)
        for (int j = 0; j < np; ++j) m = fmax(m, fabs(P[base + (size_t)j * np_max]));
    const double sc = pow2_scale(m);
    for (int j = 0; j < np_max; ++j)
        Ph[base + (size_t)j * np_max] = to_storage<S>(i < np && j < np ? P[base + (size_t)j * np_max] / sc : 0.0);
    Ps[idx] = (float)sc;
}

// Lowest-order sweep through the level's gather table (small levels): the same
// arithmetic as gs0_kernel, but each lane reads its row's target, the two element-row
// offsets and the six facet indices in three 16-byte loads, so the only dependent
// loads left are those of the matrix entries and unknowns.
template <class T, int LANES>
__global__ void __launch_bounds__(256)
gs0t_kernel(int p0, int p1, int np_max, const int *__restrict__ tbl, const T *__restrict__ A,
            const T *__restrict__ Pinv, const T *__restrict__ g, T *__restrict__ u) {
    const int lane = threadIdx.x & 31, sub = lane / LANES, t = lane % LANES;
    const int groups_per_block = blockDim.x / LANES;
    const int p = p0 + blockIdx.x * groups_per_block + (threadIdx.x / 32) * (32 / LANES) + sub;
    const bool live = p < p1;
    int e[GS0_TABLE_INTS];
#pragma unroll
    for (int i = 0; i < GS0_TABLE_INTS; ++i) e[i] = -1;
    if (live && t < np_max) {
        const int4 *rec = reinterpret_cast<const int4 *>(tbl + ((size_t)p * np_max + t) * GS0_TABLE_INTS);
#pragma unroll
        for (int v = 0; v < GS0_TABLE_INTS / 4; ++v) {
            const int4 x = rec[v];
            e[4 * v] = x.x;
            e[4 * v + 1] = x.y;
            e[4 * v + 2] = x.z;
            e[4 * v + 3] = x.w;
        }
    }
    const int row = e[0];
    T acc = 0;
    if (row >= 0) {
        acc = g[row];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const T *Ac = A + e[1 + q];
#pragma unroll
            for (int f2 = 0; f2 < 3; ++f2) {
                const int j = e[3 + 3 * q + f2];
                if (j < 0) continue;
                acc -= Ac[(2 * f2) * 2] * u[2 * (size_t)j] + Ac[(2 * f2 + 1) * 2] * u[2 * (size_t)j + 1];
            }
        }
    }
    // the valid rows of a patch are a prefix of its lane group
    const unsigned vm = __ballot_sync(0xffffffffu, row >= 0);
    const unsigned gm = LANES == 32 ? 0xffffffffu : ((1u << LANES) - 1u);
    const int np = __popc((vm >> (sub * LANES)) & gm);
    T out = 0;
    const T *Pi = live ? Pinv + (size_t)p * np_max * np_max : Pinv;
    for (int j = 0; j < np_max; ++j) {
        const T rj = __shfl_sync(0xffffffffu, acc, j, LANES);
        if (j < np && t < np) out += Pi[(size_t)j * np_max + t] * rj;
    }
    if (row >= 0) u[row] += out;
}

// ---------------------------------------------------------------- order-k sweep, TMA-staged
// One colour phase of the order-k FP32 sweep (the closed-form patch update of
// gs_kernel<float, DPF, float, true>), with the patch's matrices moved into shared
// memory by the bulk-copy engine: thread 0 posts the byte count on an mbarrier,
// then lanes of warp 0 issue one cp.async.bulk per block (the patch inverse, the
// patch's Q, and for each of the 2 nf (facet, cell) slots the coupling block of
// A_K between the facet and the cell's facet outside the patch, a contiguous
// stretch of the row-block layout).  While the copies fly, the block gathers the
// unknowns on the outside facets; it then waits on the mbarrier (bounded: after the
// wait limit it records the timeout in *flag, waits again, bounded, for its copies,
// and skips the update) and runs the residual rows and the inverse product from
// shared memory.
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, P;\n}\n"
                 : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0;
}

// polls until phase `parity` of the barrier completed or `limit_ns` of global time passed
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, unsigned long long limit_ns) {
    unsigned long long t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    while (!mbar_try_wait(bar, parity)) {
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > limit_ns) return false;
    }
    return true;
}

// SYM: the patch inverses are symmetric (generalized Stokes) and stored as packed upper
// triangles, row i holding columns i..np_max-1 at offset i np_max - i(i-1)/2, one patch every
// psz floats (psz = the packed size rounded up to 4 floats, so every copy is 16-byte sized);
// otherwise full np_max x np_max transposed inverses, of which the np used rows are copied.
//
// The patch update is taken in closed form.  With P the patch's facets and E the star's
// facets outside it (one per star cell, opposite the patch vertex), the block GS step
//   u_P <- u_P + A_PP^-1 (g - A u)_P = u_P + A_PP^-1 (g_P - A_PP u_P - A_PE u_E)
// equals A_PP^-1 (g_P - A_PE u_E), since the stored inverse is that of the assembled A_PP;
// with the AL term split off (al_split_kernel) it is A_PP^-1 (g_P - A0_PE u_E) - Q z.  So the
// kernel reads, per (facet, cell) slot, only the DPF x DPF coupling block between the slot's
// facet and the cell's outside facet (a contiguous third of the facet's row block) with its
// (0, 0) entry replaced by the AL-free one, the unknowns on the outside facets and the patch's
// Q, and overwrites u_P.
template <int DPF, bool SYM>
__global__ void __launch_bounds__(64)
gs_tma_kernel(int p0, int p1, int pf_max, int pc_max, int np_max, int psz,
              const int *__restrict__ patch_nf, const int *__restrict__ patch_facets,
              const int *__restrict__ patch_nc, const int *__restrict__ patch_cells,
              const int *__restrict__ slot_src, const int *__restrict__ patch_cint,
              const int *__restrict__ patch_cext, const double *__restrict__ cell_d,
              const float *__restrict__ A, const float *__restrict__ Pinv, const float *__restrict__ swQ,
              const float *__restrict__ swA00, const float *__restrict__ g, float *__restrict__ u, int *flag,
              unsigned long long wait_ns) {
    constexpr int NLOC = 3 * DPF;
    constexpr int BB = DPF * DPF;              // floats in one facet-pair coupling block
    extern __shared__ __align__(128) unsigned char smraw[];
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ int s_ok;
    const int p = p0 + blockIdx.x;
    if (p >= p1) return;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int nf = patch_nf[p], ncell = patch_nc[p], np = nf * DPF;
    float *Ps = reinterpret_cast<float *>(smraw);            // np rows of np_max, or psz packed
    float *As = Ps + (SYM ? (size_t)psz : (size_t)np_max * np_max);   // 2 pf_max coupling blocks
    float *Qs = As + (size_t)2 * pf_max * BB;                // pc_max columns of np_max
    float *xs = Qs + (size_t)pc_max * np_max;                // pc_max * DPF: u on the outside facets
    float *r = xs + (size_t)pc_max * DPF;                    // np_max
    float *zs = r + np_max;                                  // pc_max outside fluxes
    const uint32_t bar = smem_u32(&mbar);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_ok = 1;
    }
    __syncthreads();
    if (tid < 32) {
        const uint32_t pbytes = (uint32_t)((SYM ? psz : np * np_max) * sizeof(float));
        const uint32_t qbytes = (uint32_t)(ncell * np_max * sizeof(float));
        const uint32_t bbytes = (uint32_t)(BB * sizeof(float));
        if (tid == 0)
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                         ::"r"(bar), "r"(pbytes + qbytes + 2u * nf * bbytes) : "memory");
        __syncwarp();
        if (tid == 0) {
            const float *src = Pinv + (SYM ? (size_t)p * psz : (size_t)p * np_max * np_max);
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         ::"r"(smem_u32(Ps)), "l"(src), "r"(pbytes), "r"(bar) : "memory");
        } else if (tid == 1) {
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         ::"r"(smem_u32(Qs)), "l"(swQ + (size_t)p * pc_max * np_max), "r"(qbytes), "r"(bar)
                         : "memory");
        }
        for (int sl = tid; sl < 2 * nf; sl += 32) {
            const int src = slot_src[(size_t)p * pf_max * 2 + sl];   // slot (js, q) at js*2 + q
            const int si = src >> 2;
            const int c = patch_cells[(size_t)p * pc_max + si];
            const int e = patch_cext[(size_t)p * pc_max + si];
            const float *blk = A + (size_t)c * NLOC * NLOC + (size_t)(src & 3) * NLOC * DPF + (size_t)e * BB;
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         ::"r"(smem_u32(As + (size_t)sl * BB)), "l"(blk), "r"(bbytes), "r"(bar) : "memory");
        }
    }
    for (int t = tid; t < ncell * DPF; t += nt) {
        const int si = t / DPF, d = t % DPF;
        const int e = patch_cext[(size_t)p * pc_max + si];
        const int j = patch_cint[((size_t)p * pc_max + si) * 3 + e];
        const float x = j >= 0 ? u[(size_t)j * DPF + d] : 0.0f;
        xs[t] = x;
        if (d == 0) zs[si] = (float)cell_d[3 * (size_t)patch_cells[(size_t)p * pc_max + si] + e] * x;
    }
    // first wait: wait_ns of global time (0 = treated as expired at once, the testing hook of
    // the timeout path).  On expiry the patch update is skipped and bit 4 of *flag is set; the
    // bulk copies still target this CTA's shared memory, so the CTA keeps waiting for them in
    // bounded one-second steps (at most four) before it returns, and sets bit 8 if they still
    // have not landed (the shared memory may then be written after the CTA has exited).
    if (!(wait_ns > 0 && mbar_wait_bounded(bar, 0, wait_ns))) {
        atomicOr(flag, 4);
        s_ok = 0;
        bool drained = false;
        for (int step = 0; step < 4 && !drained; ++step) drained = mbar_wait_bounded(bar, 0, 1000000000ull);
        if (!drained) atomicOr(flag, 8);
    }
    __syncthreads();
    if (!s_ok) return;
    for (int t = tid; t < np; t += nt) {
        const int js = t / DPF, d = t % DPF;
        const int F = patch_facets[(size_t)p * pf_max + js];
        float acc = g[(size_t)F * DPF + d];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int sl = js * 2 + q;
            const int src = slot_src[(size_t)p * pf_max * 2 + sl];
            const float *Ac = As + (size_t)sl * BB + d;
            const float *xc = xs + (src >> 2) * DPF;
            acc -= (d == 0 ? swA00[(size_t)p * pf_max * 2 + sl] : Ac[0]) * xc[0];
#pragma unroll
            for (int col = 1; col < DPF; ++col) acc -= Ac[col * DPF] * xc[col];
        }
        r[t] = acc;
    }
    __syncthreads();
    for (int t = tid; t < np; t += nt) {
        float a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        int j = 0;
        if constexpr (SYM) {
            // (A_P^-1)_tj: entry (j, t) of row j for j < t, entry (t, j) of row t for j >= t
            int offc = t;                                    // offset of (j, t) while j < t
            const int offr = t * np_max - t * (t - 1) / 2 - t; // + j: offset of (t, j), j >= t
            for (; j < np; ++j) {
                const float v = Ps[j < t ? offc : offr + j];   // one load at the selected index
                offc += np_max - j - 1;
                if (j & 1) a1 += v * r[j];
                else a0 += v * r[j];
            }
        } else {
#pragma unroll 2
            for (; j + 4 <= np; j += 4) {
                a0 += Ps[(j + 0) * np_max + t] * r[j + 0];
                a1 += Ps[(j + 1) * np_max + t] * r[j + 1];
                a2 += Ps[(j + 2) * np_max + t] * r[j + 2];
                a3 += Ps[(j + 3) * np_max + t] * r[j + 3];
            }
            for (; j < np; ++j) a0 += Ps[j * np_max + t] * r[j];
        }
        for (int si = 0; si < ncell; ++si) a2 -= Qs[si * np_max + t] * zs[si];
        const int F = patch_facets[(size_t)p * pf_max + t / DPF];
        u[(size_t)F * DPF + t % DPF] = (a0 + a1) + (a2 + a3);
    }
}

// The augmented-Lagrangian split of the FP32 closed-form sweep.  The AL term of cell c is
// G_c d_c d_c^T with G_c = gamma nu_c / |K| and d_c the flux weights on the first unknown of
// each of its facets.  With z_c = d_{c,e} u_{e,0} (the outside flux through the facet e
// opposite the patch vertex), A_PE u_E = A0_PE u_E + D_P G z, so the closed form splits into
//   u_P = A_PP^-1 (g_P - A0_PE u_E) - Q z,   Q = A_PP^-1 D_P G,
// whose terms carry no O(gamma) value: Q stays bounded as gamma grows (it tends to
// A0^-1 D (D^T A0^-1 D)^+), while A_PP^-1 applied in FP32 to the O(gamma) vector D_P G z would
// lose a factor gamma of accuracy.  One block per patch writes Q (FP64 products, rounded once)
// and the (0, 0) entries of the slots' coupling blocks without the AL term.
__global__ void al_split_kernel(int n_patches, int pf_max, int pc_max, int np_max, int dpf,
                                const int *__restrict__ patch_nf, const int *__restrict__ patch_nc,
                                const int *__restrict__ patch_cells, const int *__restrict__ slot_src,
                                const int *__restrict__ patch_cext, const double *__restrict__ A,
                                const double *__restrict__ Pinv, const double *__restrict__ cell_d,
                                const double *__restrict__ cell_area, const double *__restrict__ cell_nu,
                                double nu, double gamma, float *__restrict__ Q, float *__restrict__ A00) {
    const int p = blockIdx.x;
    if (p >= n_patches) return;
    const int nf = patch_nf[p], ncell = patch_nc[p], np = nf * dpf, nloc = 3 * dpf;
    const int *ss = slot_src + (size_t)p * pf_max * 2;
    for (int sl = threadIdx.x; sl < 2 * nf; sl += blockDim.x) {
        const int si = ss[sl] >> 2, lf = ss[sl] & 3;
        const int c = patch_cells[(size_t)p * pc_max + si];
        const double G = gamma * (cell_nu ? cell_nu[c] : nu) / cell_area[c];
        const int e = patch_cext[(size_t)p * pc_max + si];
        // row 0 of facet lf, column 0 of facet e: offset lf n_loc dpf + (e dpf) dpf
        const double a = A[(size_t)c * nloc * nloc + (size_t)lf * nloc * dpf + (size_t)e * dpf * dpf];
        A00[(size_t)p * pf_max * 2 + sl] = (float)(a - G * cell_d[3 * (size_t)c + lf] * cell_d[3 * (size_t)c + e]);
    }
    const double *P = Pinv + (size_t)p * np_max * np_max;   // P[t][j] at j np_max + t
    for (int i = threadIdx.x; i < ncell * np; i += blockDim.x) {
        const int si = i / np, t = i - si * np;
        const int c = patch_cells[(size_t)p * pc_max + si];
        const double G = gamma * (cell_nu ? cell_nu[c] : nu) / cell_area[c];
        double acc = 0.0;
        for (int sl = 0; sl < 2 * nf; ++sl) {
            if ((ss[sl] >> 2) != si) continue;
            const int js = sl >> 1, lf = ss[sl] & 3;
            acc += P[(size_t)js * dpf * np_max + t] * cell_d[3 * (size_t)c + lf];
        }
        Q[((size_t)p * pc_max + si) * np_max + t] = (float)(G * acc);
    }
}

// packed symmetric FP32 copy of the order-k patch inverses (symmetric operators only): the
// upper triangle of (P + P^T)/2 from the FP64 inverses, rounded once; one block per patch
__global__ void pack_sym_kernel(int n_patches, int np_max, int psz, const double *__restrict__ Pinv,
                                float *__restrict__ out) {
    const int p = blockIdx.x;
    if (p >= n_patches) return;
    const double *P = Pinv + (size_t)p * np_max * np_max;
    float *o = out + (size_t)p * psz;
    for (int e = threadIdx.x; e < np_max * np_max; e += blockDim.x) {
        const int i = e / np_max, j = e % np_max;
        if (j < i) continue;
        o[i * np_max - i * (i - 1) / 2 + (j - i)] = (float)(0.5 * (P[(size_t)i * np_max + j] + P[(size_t)j * np_max + i]));
    }
    const int used = np_max * (np_max + 1) / 2;
    for (int e = used + threadIdx.x; e < psz; e += blockDim.x) o[e] = 0.0f;
}

// Lowest-order sweep (DPF = 2): LANES consecutive lanes of a warp own one patch
// (row t of the patch on lane t, np <= LANES <= 32), so a 256-thread block works on
// 256/LANES patches at once instead of one; the block inverse is applied with
// shuffles inside the lane group, without shared memory.
template <class T, int LANES>
__global__ void __launch_bounds__(256)
gs0_kernel(int p0, int p1, int pf_max, int pc_max, int np_max, const int *__restrict__ patch_nf,
           const int *__restrict__ patch_facets, const int *__restrict__ patch_cells,
           const int *__restrict__ slot_src, const int *__restrict__ cell_int, const T *__restrict__ A,
           const T *__restrict__ Pinv, const T *__restrict__ g, T *__restrict__ u) {
    const int lane = threadIdx.x & 31, sub = lane / LANES, t = lane % LANES;
    const int groups_per_block = blockDim.x / LANES;
    const int p = p0 + blockIdx.x * groups_per_block + (threadIdx.x / 32) * (32 / LANES) + sub;
    const bool live = p < p1;
    const int np = live ? 2 * patch_nf[p] : 0;
    T acc = 0;
    int F = -1;
    if (t < np) {
        const int js = t >> 1, d = t & 1;
        F = patch_facets[(size_t)p * pf_max + js];
        acc = g[2 * (size_t)F + d];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int src = slot_src[((size_t)p * pf_max + js) * 2 + q];
            const int c = patch_cells[(size_t)p * pc_max + (src >> 2)];
            const int lf = src & 3;
            const T *Ac = A + (size_t)c * 36 + lf * 12 + d;
#pragma unroll
            for (int f2 = 0; f2 < 3; ++f2) {
                const int j = cell_int[3 * c + f2];
                if (j < 0) continue;
                acc -= Ac[(2 * f2) * 2] * u[2 * (size_t)j] + Ac[(2 * f2 + 1) * 2] * u[2 * (size_t)j + 1];
            }
        }
    }
    // u_s += A_ss^{-1} r_s: lane t forms row t from the group's residuals (every lane of the
    // warp runs the same np_max shuffles; width LANES keeps them inside the group)
    T out = 0;
    const T *Pi = live ? Pinv + (size_t)p * np_max * np_max : Pinv;
    for (int j = 0; j < np_max; ++j) {
        const T rj = __shfl_sync(0xffffffffu, acc, j, LANES);
        if (j < np && t < np) out += Pi[(size_t)j * np_max + t] * rj;
    }
    if (t < np) u[2 * (size_t)F + (t & 1)] += out;
}

template <class T>
__global__ void hp_restrict_kernel(int k, int64_t n_int, const T *r, T *r0) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_int) return;
    int dpf = 2 * (k + 1);
    r0[2 * i] = r[i * dpf];
    r0[2 * i + 1] = r[i * dpf + k + 1];
}

template <class T>
__global__ void hp_prolong_kernel(int k, int64_t n_int, const T *d0, T *u) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_int) return;
    int dpf = 2 * (k + 1);
    u[i * dpf] += d0[2 * i];
    u[i * dpf + k + 1] += d0[2 * i + 1];
}

template <class T>
__global__ void prolong_B_kernel(int64_t nB, const int *__restrict__ fineB,
                                 const int *__restrict__ fineB_src, const int *__restrict__ ccell_int,
                                 const T *__restrict__ W, const T *__restrict__ uc, T *__restrict__ tmp,
                                 T *__restrict__ uf) {
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nB) return;
    T v0 = 0, v1 = 0;
    for (int q = 0; q < 2; ++q) {
        int src = fineB_src[2 * b + q];
        int P = src >> 4, s = src & 15;
        const T *Wk = W + (size_t)P * 72;
        for (int fp = 0; fp < 3; ++fp) {
            int j = ccell_int[3 * P + fp];
            if (j < 0) continue;
            for (int cq = 0; cq < 2; ++cq) {
                T u = uc[2 * (size_t)j + cq];
                v0 += Wk[(2 * s) * 6 + 2 * fp + cq] * u;
                v1 += Wk[(2 * s + 1) * 6 + 2 * fp + cq] * u;
            }
        }
    }
    int i = fineB[b];
    tmp[2 * (size_t)i] = v0;
    tmp[2 * (size_t)i + 1] = v1;
    uf[2 * (size_t)i] += v0;
    uf[2 * (size_t)i + 1] += v1;
}

template <class T>
__global__ void prolong_T_kernel(int64_t ncc, const int *__restrict__ slots, const T *__restrict__ H,
                                 const T *__restrict__ tmp, T *__restrict__ uf) {
    int64_t P = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (P >= ncc) return;
    T b[12];
    for (int s = 0; s < 6; ++s) {
        int i = slots[9 * P + s];
        b[2 * s] = i >= 0 ? tmp[2 * (size_t)i] : T(0);
        b[2 * s + 1] = i >= 0 ? tmp[2 * (size_t)i + 1] : T(0);
    }
    const T *Hk = H + (size_t)P * 72;
    for (int t = 0; t < 6; ++t) {
        T acc = 0;
        for (int c = 0; c < 12; ++c) acc += Hk[t * 12 + c] * b[c];
        int i = slots[9 * P + 6 + t / 2];
        uf[2 * (size_t)i + (t & 1)] += acc;
    }
}

template <class T>
__global__ void restrict_T_kernel(int64_t ncc, const int *__restrict__ slots, const T *__restrict__ H,
                                  const T *__restrict__ rf, T *__restrict__ t1) {
    int64_t P = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (P >= ncc) return;
    T rT[6];
    for (int t = 0; t < 6; ++t) rT[t] = rf[2 * (size_t)slots[9 * P + 6 + t / 2] + (t & 1)];
    const T *Hk = H + (size_t)P * 72;
    for (int c = 0; c < 12; ++c) {
        T acc = 0;
        for (int t = 0; t < 6; ++t) acc += Hk[t * 12 + c] * rT[t];
        t1[12 * P + c] = acc;
    }
}

template <class T>
__global__ void restrict_B_kernel(int64_t ncc, const int *__restrict__ slots, const int *__restrict__ nbr,
                                  const T *__restrict__ W, const T *__restrict__ rf,
                                  const T *__restrict__ t1, T *__restrict__ t2) {
    int64_t P = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (P >= ncc) return;
    T z[12];
    for (int s = 0; s < 6; ++s) {
        int i = slots[9 * P + s];
        if (i < 0) {
            z[2 * s] = z[2 * s + 1] = 0;
            continue;
        }
        int nb = nbr[6 * P + s];
        int Q = nb >> 4, s2 = nb & 15;
        for (int c = 0; c < 2; ++c)
            z[2 * s + c] = rf[2 * (size_t)i + c] + t1[12 * P + 2 * s + c] + t1[12 * (size_t)Q + 2 * s2 + c];
    }
    const T *Wk = W + (size_t)P * 72;
    for (int col = 0; col < 6; ++col) {
        T acc = 0;
        for (int row = 0; row < 12; ++row) acc += Wk[row * 6 + col] * z[row];
        t2[6 * P + col] = acc;
    }
}

template <class T>
__global__ void restrict_C_kernel(int64_t n_int_c, const int *__restrict__ facet_adj_c,
                                  const T *__restrict__ t2, T *__restrict__ rc) {
    int64_t G = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (G >= n_int_c) return;
    T a0 = 0, a1 = 0;
    for (int q = 0; q < 2; ++q) {
        int adj = facet_adj_c[2 * G + q];
        int K = adj >> 2, lf = adj & 3;
        a0 += t2[6 * (size_t)K + 2 * lf];
        a1 += t2[6 * (size_t)K + 2 * lf + 1];
    }
    rc[2 * G] = a0;
    rc[2 * G + 1] = a1;
}

__global__ void coarse_apply_kernel(const double *__restrict__ inv, int64_t n,
                                    const double *__restrict__ g, double *__restrict__ u) {
    int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
    int lane = threadIdx.x & 31;
    if (row >= n) return;
    double acc = 0.0;
    for (int64_t j = lane; j < n; j += 32) acc += inv[row * n + j] * g[j];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) u[row] = acc;
}

__global__ void d2f_kernel(const double *x, float *y, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] = (float)x[i];
}
__global__ void f2d_kernel(const float *x, double *y, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] = (double)x[i];
}
template <class T>
__global__ void fill_kernel(T *x, T v, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) x[i] = v;
}
__global__ void axpby_kernel(double a, const double *x, double b, double *y, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] = a * x[i] + b * y[i];
}

// ---------------------------------------------------------------- Krylov
__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// block-reduce acc[0..nv) (warp shuffles, then one shared-memory pass) and
// write partials[i*gridDim.x + block]
template <int NVB>
__device__ void block_reduce_store(const double *acc, int nv, double *partials) {
    __shared__ double red[KRYLOV_THREADS / 32][NVB];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NVB; ++i) {
        if (i < nv) {
            double v = warp_sum(acc[i]);
            if (lane == 0) red[wid][i] = v;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nv; i += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < KRYLOV_THREADS / 32; ++w) s += red[w][i];
        partials[(size_t)i * gridDim.x + blockIdx.x] = s;
    }
}

// partials of h_i = <V_i, w> for the vectors i0 = 16*blockIdx.y .. i0+nvb-1 (nvb <= NVB <= 16);
// one register accumulator per vector, w read once per chunk of vectors
template <int NVB>
__global__ void __launch_bounds__(KRYLOV_THREADS)
dots_kernel(const double *__restrict__ V, int nv, int64_t ld, const double *__restrict__ w, int64_t n,
            double *__restrict__ partials) {
    const int i0 = 16 * blockIdx.y;
    const int nvb = min(nv - i0, NVB);
    const double *Vb = V + (size_t)i0 * ld;
    double acc[NVB];
#pragma unroll
    for (int i = 0; i < NVB; ++i) acc[i] = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const double we = w[e];
#pragma unroll
        for (int i = 0; i < NVB; ++i)
            if (i < nvb) acc[i] = fma(Vb[(size_t)i * ld + e], we, acc[i]);
    }
    block_reduce_store<NVB>(acc, nvb, partials + (size_t)i0 * gridDim.x);
}

// w -= Σ_{i<nv} h_i V_i; MODE 1: also partials of <V_i, w_new> (nv <= NVB <= 16, the basis
// values held in registers between the two); MODE 2: partials of <w_new, w_new>; MODE 0: update only
template <int NVB, int MODE>
__global__ void __launch_bounds__(KRYLOV_THREADS)
update_dots_kernel(const double *__restrict__ V, int nv, int64_t ld, double *__restrict__ w, int64_t n,
                   const double *__restrict__ h, double *__restrict__ partials) {
    __shared__ double hs[MAXV];
    for (int i = threadIdx.x; i < nv; i += blockDim.x) hs[i] = h[i];
    __syncthreads();
    constexpr int NA = MODE == 1 ? NVB : 1;
    double acc[NA];
#pragma unroll
    for (int i = 0; i < NA; ++i) acc[i] = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        double we = w[e];
        if (MODE == 1 && NVB <= 16) {
            // basis values stay in registers between the update and the dots
            double vr[NVB];
#pragma unroll
            for (int i = 0; i < NVB; ++i) vr[i] = i < nv ? V[(size_t)i * ld + e] : 0.0;
#pragma unroll
            for (int i = 0; i < NVB; ++i)
                if (i < nv) we = fma(-hs[i], vr[i], we);
            w[e] = we;
#pragma unroll
            for (int i = 0; i < NVB; ++i)
                if (i < nv) acc[i] = fma(vr[i], we, acc[i]);
        } else if (MODE == 1) {
            // too many for registers: the second read of V_i(e) is served by L1
#pragma unroll
            for (int i = 0; i < NVB; ++i)
                if (i < nv) we = fma(-hs[i], V[(size_t)i * ld + e], we);
            w[e] = we;
#pragma unroll
            for (int i = 0; i < NVB; ++i)
                if (i < nv) acc[i] = fma(V[(size_t)i * ld + e], we, acc[i]);
        } else {
#pragma unroll 4
            for (int i = 0; i < nv; ++i) we = fma(-hs[i], V[(size_t)i * ld + e], we);
            w[e] = we;
            if (MODE == 2) acc[0] = fma(we, we, acc[0]);
        }
    }
    if (MODE != 0) block_reduce_store<NA>(acc, MODE == 1 ? nv : 1, partials);
}

__global__ void reduce_partials_kernel(const double *__restrict__ partials, int nv, int nb,
                                       double *__restrict__ out, int accumulate) {
    int i = blockIdx.x;
    if (i >= nv) return;
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += 32) s += partials[(size_t)i * nb + b];
    s = warp_sum(s);
    if (threadIdx.x == 0) out[i] = accumulate ? out[i] + s : s;
}

__global__ void givens_kernel(double *sm, int j, int R) {
    SmallLayout Ly{R};
    double *H = sm + Ly.H(), *cs = sm + Ly.cs(), *sn = sm + Ly.sn(), *g = sm + Ly.g();
    double col[MAXV + 1];
    for (int i = 0; i <= j; ++i) col[i] = sm[Ly.h1() + i] + sm[Ly.h2() + i];
    double hn = sqrt(fmax(sm[Ly.nrm2()], 0.0));
    col[j + 1] = hn;
    for (int i = 0; i < j; ++i) {
        double a = col[i], b = col[i + 1];
        col[i] = cs[i] * a + sn[i] * b;
        col[i + 1] = -sn[i] * a + cs[i] * b;
    }
    double den = hypot(col[j], col[j + 1]);
    double c = den > 0.0 ? col[j] / den : 1.0, s = den > 0.0 ? col[j + 1] / den : 0.0;
    cs[j] = c;
    sn[j] = s;
    col[j] = den;
    col[j + 1] = 0.0;
    g[j + 1] = -s * g[j];
    g[j] = c * g[j];
    for (int i = 0; i <= j + 1; ++i) H[(size_t)j * (R + 1) + i] = col[i];
    sm[Ly.res()] = fabs(g[j + 1]);
    sm[Ly.hn()] = hn;
}

__global__ void scale_next_kernel(const double *__restrict__ w, double *__restrict__ v, int64_t n,
                                  const double *__restrict__ sm, int hn_off) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double hn = sm[hn_off];
    if (i < n) v[i] = hn > 0.0 ? w[i] / hn : 0.0;
}

__global__ void init_cycle_kernel(const double *__restrict__ r, double *__restrict__ v0, int64_t n,
                                  double *__restrict__ sm, int R) {
    SmallLayout Ly{R};
    double beta = sqrt(fmax(sm[Ly.nrm2()], 0.0));
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) v0[i] = beta > 0.0 ? r[i] / beta : 0.0;
    if (i <= R) sm[Ly.g() + i] = (i == 0) ? beta : 0.0;
}

__global__ void backsolve_kernel(double *sm, int m, int R) {
    SmallLayout Ly{R};
    const double *H = sm + Ly.H(), *g = sm + Ly.g();
    double *y = sm + Ly.y();
    for (int i = m - 1; i >= 0; --i) {
        double s = g[i];
        for (int p = i + 1; p < m; ++p) s -= H[(size_t)p * (R + 1) + i] * y[p];
        y[i] = s / H[(size_t)i * (R + 1) + i];
    }
}

__global__ void update_x_kernel(const double *__restrict__ Z, int m, int64_t ld, const double *__restrict__ sm,
                                int y_off, double *__restrict__ x, int64_t n) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    double s = x[e];
    for (int j = 0; j < m; ++j) s += sm[y_off + j] * Z[(size_t)j * ld + e];
    x[e] = s;
}

// ---------------------------------------------------------------- Uzawa
__global__ void uzawa_rhs_kernel(int64_t n_int, int dpf, int nfc, const int *__restrict__ facet_adj,
                                 const double *__restrict__ cell_d, const double *__restrict__ F,
                                 const double *__restrict__ p, double *__restrict__ g) {
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n_int * dpf) return;
    int64_t i = idx / dpf;
    int d = (int)(idx - i * dpf);
    double v = F[idx];
    if (d == 0)
        for (int q = 0; q < 2; ++q) {
            int adj = facet_adj[2 * i + q];
            if (adj < 0) continue;
            int c = adj >> 2, lf = adj & 3;
            v += p[c] * cell_d[nfc * c + lf];
        }
    g[idx] = v;
}

__global__ void __launch_bounds__(KRYLOV_THREADS)
uzawa_update_kernel(int64_t nc, int dpf, int nfc, const int *__restrict__ cell_int,
                    const double *__restrict__ cell_d, const double *__restrict__ area,
                    const double *__restrict__ u, double *__restrict__ p, double gamma, double nu,
                    const double *__restrict__ nu_cell, const double *__restrict__ bflux,
                    double *__restrict__ partials) {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc;
         c += (int64_t)gridDim.x * blockDim.x) {
        double du = 0.0;
        for (int f = 0; f < nfc; ++f) {
            int j = cell_int[nfc * c + f];
            if (j >= 0) du += cell_d[nfc * c + f] * u[(size_t)j * dpf];
        }
        if (bflux) du += bflux[c];   // flux of inhomogeneous Dirichlet data
        double a = area[c];
        double dp = gamma * (nu_cell ? nu_cell[c] : nu) * du / a;
        double pn = p[c] - dp;
        p[c] = pn;
        acc[0] += a * dp * dp;
        acc[1] += a * pn * pn;
        acc[2] += du * du;
        acc[3] += du * du / a;   // |div u_h|^2 on the cell: div u_h is the constant du / |K|
    }
    block_reduce_store<4>(acc, 4, partials);
}

template <class T>
cudaError_t apply_dispatch(const DevLevel &L, int dpf, const T *A, const T *x, const T *g, T *y,
                           cudaStream_t s) {
    int64_t n = L.n_int * dpf;
    if (n == 0) return cudaSuccess;
    unsigned nb = blocks_for(n, 256);
    switch (dpf) {
    case 2: note_launches(1); apply_kernel<T, 2><<<nb, 256, 0, s>>>(L.n_int, L.facet_adj.p, L.cell_int.p, A, nullptr, x, g, y); break;
    case 4: note_launches(1); apply_kernel<T, 4><<<nb, 256, 0, s>>>(L.n_int, L.facet_adj.p, L.cell_int.p, A, nullptr, x, g, y); break;
    case 6: note_launches(1); apply_kernel<T, 6><<<nb, 256, 0, s>>>(L.n_int, L.facet_adj.p, L.cell_int.p, A, nullptr, x, g, y); break;
    case 8: note_launches(1); apply_kernel<T, 8><<<nb, 256, 0, s>>>(L.n_int, L.facet_adj.p, L.cell_int.p, A, nullptr, x, g, y); break;
    case 10: note_launches(1); apply_kernel<T, 10><<<nb, 256, 0, s>>>(L.n_int, L.facet_adj.p, L.cell_int.p, A, nullptr, x, g, y); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int DPF, bool SYM>
size_t tma_sweep_smem(const DevLevel &L, const DevOperator &op) {
    const size_t bb = (size_t)DPF * DPF;         // one facet-pair coupling block
    const size_t pin = SYM ? (size_t)packed_patch_size(op.np_max) : (size_t)op.np_max * op.np_max;
    return sizeof(float) * (pin + 2 * (size_t)L.pf_max * bb + (size_t)L.pc_max * op.np_max +
                            (size_t)L.pc_max * DPF + op.np_max + L.pc_max);
}

// the bulk copies need 16-byte aligned sources, destinations and sizes: the patch
// inverse (np_max² floats, rows of np_max; or the packed triangle, psz floats), the
// coupling blocks (DPF² floats, at offsets of multiples of DPF² floats), Q (columns of
// np_max floats) and both bases
template <int DPF, bool SYM>
bool tma_sweep_ok(const DevLevel &L, const DevOperator &op, const float *A, const float *Pinv) {
    const size_t smem = tma_sweep_smem<DPF, SYM>(L, op);
    if ((op.np_max * sizeof(float)) % 16 || ((size_t)op.np_max * op.np_max * sizeof(float)) % 16 ||
        (packed_patch_size(op.np_max) * sizeof(float)) % 16 || (DPF * DPF * sizeof(float)) % 16)
        return false;
    if (!L.patch_cint.p || !L.patch_cext.p || !op.swQ.p || !op.swA00.p) return false;
    if (reinterpret_cast<uintptr_t>(A) % 16 || reinterpret_cast<uintptr_t>(Pinv) % 16) return false;
    if (smem > 100 * 1024) return false;
    if (cudaFuncSetAttribute(gs_tma_kernel<DPF, SYM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}

template <class T, int DPF>
cudaError_t gs_launch(const DevLevel &L, const DevOperator &op, const T *A, const T *Pinv, int colour,
                      const T *g, T *u, cudaStream_t s) {
    int p0 = L.colour_ptr[colour], p1 = L.colour_ptr[colour + 1];
    if (p1 <= p0) return cudaSuccess;
    if (DPF == 2 && op.np_max <= 32) {
        // lowest order: lane groups of 16 (or 32) per patch, 256-thread blocks
        note_launches(1);
        const int lanes = op.np_max <= 16 ? 16 : 32;
        const int per_block = 256 / lanes;
        const unsigned nb = (unsigned)((p1 - p0 + per_block - 1) / per_block);
        // the gather table pays off in FP32 (about 4% of the mixed solve at 512x512); with FP64
        // values the table-driven kernel measured slower than the index-chasing one
        if (std::is_same<T, float>::value && lanes == 16 && L.gs0_table.p && op.np_max == 2 * L.pf_max)
            gs0t_kernel<T, 16><<<nb, 256, 0, s>>>(p0, p1, op.np_max, L.gs0_table.p, A, Pinv, g, u);
        else if (lanes == 16)
            gs0_kernel<T, 16><<<nb, 256, 0, s>>>(p0, p1, L.pf_max, L.pc_max, op.np_max, L.patch_nf.p,
                                                 L.patch_facets.p, L.patch_cells.p, L.patch_slot_src.p,
                                                 L.cell_int.p, A, Pinv, g, u);
        else
            gs0_kernel<T, 32><<<nb, 256, 0, s>>>(p0, p1, L.pf_max, L.pc_max, op.np_max, L.patch_nf.p,
                                                 L.patch_facets.p, L.patch_cells.p, L.patch_slot_src.p,
                                                 L.cell_int.p, A, Pinv, g, u);
        return cudaGetLastError();
    }
    int nt = ((op.np_max + 31) / 32) * 32;
    if (nt > 256) nt = 256;
    if (nt < 32) nt = 32;
    if constexpr (std::is_same<T, float>::value && DPF >= 4) {
        // symmetric operators sweep with the packed inverses when this is the operator's own
        // FP32 copy (half the inverse bytes); otherwise the full transposed inverses
        const bool sym = op.Pinvp.p && Pinv == op.Pinvf.p && A == op.Af.p;
        if (op.tma_flag && nt == 64 && sym && tma_sweep_ok<DPF, true>(L, op, A, op.Pinvp.p)) {
            const size_t tsm = tma_sweep_smem<DPF, true>(L, op);
            note_launches(1);
            gs_tma_kernel<DPF, true><<<p1 - p0, 64, tsm, s>>>(
                p0, p1, L.pf_max, L.pc_max, op.np_max, packed_patch_size(op.np_max), L.patch_nf.p, L.patch_facets.p,
                L.patch_nc.p, L.patch_cells.p, L.patch_slot_src.p, L.patch_cint.p, L.patch_cext.p, L.cell_d.p, A,
                op.Pinvp.p, op.swQ.p, op.swA00.p, g, u, op.tma_flag, op.tma_wait_ns);
            return cudaGetLastError();
        }
        if (op.tma_flag && nt == 64 && A == op.Af.p && Pinv == op.Pinvf.p &&
            tma_sweep_ok<DPF, false>(L, op, A, Pinv)) {
            const size_t tsm = tma_sweep_smem<DPF, false>(L, op);
            note_launches(1);
            gs_tma_kernel<DPF, false><<<p1 - p0, 64, tsm, s>>>(
                p0, p1, L.pf_max, L.pc_max, op.np_max, 0, L.patch_nf.p, L.patch_facets.p, L.patch_nc.p,
                L.patch_cells.p, L.patch_slot_src.p, L.patch_cint.p, L.patch_cext.p, L.cell_d.p, A, Pinv, op.swQ.p,
                op.swA00.p, g, u, op.tma_flag, op.tma_wait_ns);
            return cudaGetLastError();
        }
    }
    // closed form where the level has the outside-facet table: FP64 directly, FP32 with the AL
    // split of its own matrices (otherwise the correction form)
    const bool fp32 = std::is_same<T, float>::value;
    const bool own = (const void *)A == (const void *)op.Af.p && (const void *)Pinv == (const void *)op.Pinvf.p;
    note_launches(1);
    if (L.patch_cext.p && (!fp32 || (own && op.swQ.p && op.swA00.p))) {
        const size_t smem = sizeof(T) * ((size_t)L.pc_max * DPF + op.np_max + L.pc_max);
        gs_kernel<T, DPF, T, true><<<p1 - p0, nt, smem, s>>>(
            p0, p1, L.pf_max, L.pc_max, op.np_max, L.patch_nf.p, L.patch_facets.p, L.patch_nc.p, L.patch_cells.p,
            L.patch_slot_src.p, L.cell_int.p, L.patch_cext.p, fp32 ? op.swQ.p : nullptr,
            fp32 ? op.swA00.p : nullptr, L.cell_d.p, A, nullptr, Pinv, nullptr, g, u);
    } else {
        const size_t smem = sizeof(T) * ((size_t)L.pc_max * 3 * DPF + op.np_max + L.pc_max);
        gs_kernel<T, DPF><<<p1 - p0, nt, smem, s>>>(p0, p1, L.pf_max, L.pc_max, op.np_max, L.patch_nf.p,
                                                    L.patch_facets.p, L.patch_nc.p, L.patch_cells.p,
                                                    L.patch_slot_src.p, L.cell_int.p, nullptr, nullptr, nullptr,
                                                    nullptr, A, nullptr, Pinv, nullptr, g, u);
    }
    return cudaGetLastError();
}

template <class S, int DPF>
cudaError_t gs_launch_h(const DevLevel &L, const DevOperator &op, int colour, const float *g, float *u,
                        cudaStream_t s) {
    int p0 = L.colour_ptr[colour], p1 = L.colour_ptr[colour + 1];
    if (p1 <= p0) return cudaSuccess;
    int nt = ((op.np_max + 31) / 32) * 32;
    if (nt > 256) nt = 256;
    if (nt < 32) nt = 32;
    // the 16-bit copies keep the correction form: their rounding model (u + P (g - A u) with
    // the rounded matrices) is the one the 16-bit precisions are defined by
    const size_t smem = sizeof(float) * ((size_t)L.pc_max * 3 * DPF + op.np_max + L.pc_max);
    note_launches(1);
    gs_kernel<float, DPF, S><<<p1 - p0, nt, smem, s>>>(
        p0, p1, L.pf_max, L.pc_max, op.np_max, L.patch_nf.p, L.patch_facets.p, L.patch_nc.p, L.patch_cells.p,
        L.patch_slot_src.p, L.cell_int.p, nullptr, nullptr, nullptr, nullptr, reinterpret_cast<const S *>(op.Ah.p),
        op.Ah_s.p, reinterpret_cast<const S *>(op.Pinvh.p), op.Pinvh_s.p, g, u);
    return cudaGetLastError();
}

template <class S, int DPF>
cudaError_t apply_launch_h(const DevLevel &L, const DevOperator &op, const float *x, const float *g, float *y,
                           cudaStream_t s) {
    const int64_t n = L.n_int * DPF;
    if (n == 0) return cudaSuccess;
    note_launches(1);
    apply_kernel<float, DPF, S><<<blocks_for(n, 256), 256, 0, s>>>(
        L.n_int, L.facet_adj.p, L.cell_int.p, reinterpret_cast<const S *>(op.Ah.p), op.Ah_s.p, x, g, y);
    return cudaGetLastError();
}

template <class S>
cudaError_t round16_launch(const DevLevel &L, DevOperator &op, cudaStream_t s) {
    const int64_t nrow = L.nc * op.nloc;
    note_launches(1);
    switch (op.dpf) {
    case 2: round_element_rows_kernel<S, 2><<<blocks_for(nrow, 128), 128, 0, s>>>(L.nc, op.A.p, reinterpret_cast<S *>(op.Ah.p), op.Ah_s.p); break;
    case 4: round_element_rows_kernel<S, 4><<<blocks_for(nrow, 128), 128, 0, s>>>(L.nc, op.A.p, reinterpret_cast<S *>(op.Ah.p), op.Ah_s.p); break;
    case 6: round_element_rows_kernel<S, 6><<<blocks_for(nrow, 128), 128, 0, s>>>(L.nc, op.A.p, reinterpret_cast<S *>(op.Ah.p), op.Ah_s.p); break;
    case 8: round_element_rows_kernel<S, 8><<<blocks_for(nrow, 128), 128, 0, s>>>(L.nc, op.A.p, reinterpret_cast<S *>(op.Ah.p), op.Ah_s.p); break;
    case 10: round_element_rows_kernel<S, 10><<<blocks_for(nrow, 128), 128, 0, s>>>(L.nc, op.A.p, reinterpret_cast<S *>(op.Ah.p), op.Ah_s.p); break;
    default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || L.n_patches == 0) return e;
    const int64_t nprow = (int64_t)L.n_patches * op.np_max;
    note_launches(1);
    round_patch_rows_kernel<S><<<blocks_for(nprow, 128), 128, 0, s>>>(
        L.n_patches, op.np_max, op.dpf, L.patch_nf.p, op.Pinv.p, reinterpret_cast<S *>(op.Pinvh.p), op.Pinvh_s.p);
    return cudaGetLastError();
}

} // namespace

cudaError_t launch_al_split(const DevLevel &L, DevOperator &op, double nu, const double *cell_nu, double gamma,
                            cudaStream_t s) {
    if (L.n_patches == 0 || !L.patch_cext.p) return cudaSuccess;
    const size_t nq = (size_t)L.n_patches * L.pc_max * op.np_max;
    if (!op.swQ.p || op.swQ.n < nq || !op.swA00.p || op.swA00.n < (size_t)L.n_patches * L.pf_max * 2)
        return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(op.swQ.p, 0, sizeof(float) * nq, s);
    if (e != cudaSuccess) return e;
    note_launches(1);
    al_split_kernel<<<L.n_patches, 128, 0, s>>>(L.n_patches, L.pf_max, L.pc_max, op.np_max, op.dpf, L.patch_nf.p,
                                                L.patch_nc.p, L.patch_cells.p, L.patch_slot_src.p, L.patch_cext.p,
                                                op.A.p, op.Pinv.p, L.cell_d.p, L.cell_area.p, cell_nu, nu, gamma,
                                                op.swQ.p, op.swA00.p);
    return cudaGetLastError();
}

cudaError_t launch_pack_sym(const DevLevel &L, DevOperator &op, cudaStream_t s) {
    if (L.n_patches == 0) return cudaSuccess;
    note_launches(1);
    pack_sym_kernel<<<L.n_patches, 256, 0, s>>>(L.n_patches, op.np_max, packed_patch_size(op.np_max), op.Pinv.p,
                                                op.Pinvp.p);
    return cudaGetLastError();
}

cudaError_t launch_round16(const DevLevel &L, DevOperator &op, int fmt, cudaStream_t s) {
    if (fmt == HDG_MIXED_BF16) return round16_launch<__nv_bfloat16>(L, op, s);
    if (fmt == HDG_MIXED_FP16) return round16_launch<__half>(L, op, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_apply_h(const DevLevel &L, const DevOperator &op, const float *x, const float *g, float *y,
                           cudaStream_t s) {
    const bool bf = op.h_fmt == HDG_MIXED_BF16;
    if (!bf && op.h_fmt != HDG_MIXED_FP16) return cudaErrorInvalidValue;
    switch (op.dpf) {
#define HDG_APPLY_H(D) \
    case D: return bf ? apply_launch_h<__nv_bfloat16, D>(L, op, x, g, y, s) : apply_launch_h<__half, D>(L, op, x, g, y, s);
    HDG_APPLY_H(2) HDG_APPLY_H(4) HDG_APPLY_H(6) HDG_APPLY_H(8) HDG_APPLY_H(10)
#undef HDG_APPLY_H
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_gs_colour_h(const DevLevel &L, const DevOperator &op, int colour, const float *g, float *u,
                               cudaStream_t s) {
    const bool bf = op.h_fmt == HDG_MIXED_BF16;
    if (!bf && op.h_fmt != HDG_MIXED_FP16) return cudaErrorInvalidValue;
    switch (op.dpf) {
#define HDG_GS_H(D) \
    case D: return bf ? gs_launch_h<__nv_bfloat16, D>(L, op, colour, g, u, s) : gs_launch_h<__half, D>(L, op, colour, g, u, s);
    HDG_GS_H(2) HDG_GS_H(4) HDG_GS_H(6) HDG_GS_H(8) HDG_GS_H(10)
#undef HDG_GS_H
    default: return cudaErrorInvalidValue;
    }
}

template <class T>
cudaError_t launch_apply(const DevLevel &L, const DevOperator &op, const T *A, const T *x, const T *g,
                         T *y, cudaStream_t s) {
    if (L.dim == 3) return launch_apply3<T>(L, op.dpf, A, x, g, y, s);
    return apply_dispatch<T>(L, op.dpf, A, x, g, y, s);
}

template <class T>
cudaError_t launch_gs_colour(const DevLevel &L, const DevOperator &op, const T *A, const T *Pinv,
                             int colour, const T *g, T *u, cudaStream_t s) {
    if (L.dim == 3) return launch_gs_colour3<T>(L, op, A, Pinv, colour, g, u, s);
    switch (op.dpf) {
    case 2: return gs_launch<T, 2>(L, op, A, Pinv, colour, g, u, s);
    case 4: return gs_launch<T, 4>(L, op, A, Pinv, colour, g, u, s);
    case 6: return gs_launch<T, 6>(L, op, A, Pinv, colour, g, u, s);
    case 8: return gs_launch<T, 8>(L, op, A, Pinv, colour, g, u, s);
    case 10: return gs_launch<T, 10>(L, op, A, Pinv, colour, g, u, s);
    default: return cudaErrorInvalidValue;
    }
}

template <class T>
cudaError_t launch_prolong_add(const DevLevel &F, const DevLevel &C, const T *W, const T *Hm, const T *uc,
                               T *tmp, T *uf, cudaStream_t s) {
    if (F.dim == 3) return launch_prolong_add3<T>(F, C, W, Hm, uc, tmp, uf, s);
    if (F.nB > 0) {
        note_launches(1);
        prolong_B_kernel<T><<<blocks_for(F.nB, 128), 128, 0, s>>>(F.nB, F.tr_fineB.p, F.tr_fineB_src.p,
                                                                 C.cell_int.p, W, uc, tmp, uf);
    }
    if (F.nc_coarse > 0) {
        note_launches(1);
        prolong_T_kernel<T><<<blocks_for(F.nc_coarse, 128), 128, 0, s>>>(F.nc_coarse, F.tr_slots.p, Hm,
                                                                         tmp, uf);
    }
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_restrict(const DevLevel &F, const DevLevel &C, const T *W, const T *Hm, const T *rf,
                            T *t1, T *t2, T *rc, cudaStream_t s) {
    if (F.dim == 3) return launch_restrict3<T>(F, C, W, Hm, rf, t1, t2, rc, s);
    if (F.nc_coarse > 0) {
        note_launches(1);
        restrict_T_kernel<T><<<blocks_for(F.nc_coarse, 128), 128, 0, s>>>(F.nc_coarse, F.tr_slots.p, Hm,
                                                                          rf, t1);
        note_launches(1);
        restrict_B_kernel<T><<<blocks_for(F.nc_coarse, 128), 128, 0, s>>>(F.nc_coarse, F.tr_slots.p,
                                                                          F.tr_nbr.p, W, rf, t1, t2);
    }
    if (C.n_int > 0) {
        note_launches(1);
        restrict_C_kernel<T><<<blocks_for(C.n_int, 128), 128, 0, s>>>(C.n_int, C.facet_adj.p, t2, rc);
    }
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_hp_restrict(int k, int64_t n_int, const T *r, T *r0, cudaStream_t s) {
    if (n_int == 0) return cudaSuccess;
    note_launches(1);
    hp_restrict_kernel<T><<<blocks_for(n_int, 256), 256, 0, s>>>(k, n_int, r, r0);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_hp_prolong_add(int k, int64_t n_int, const T *d0, T *u, cudaStream_t s) {
    if (n_int == 0) return cudaSuccess;
    note_launches(1);
    hp_prolong_kernel<T><<<blocks_for(n_int, 256), 256, 0, s>>>(k, n_int, d0, u);
    return cudaGetLastError();
}

cudaError_t launch_coarse_apply(const double *inv, int64_t n, const double *g, double *u, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    note_launches(1);
    coarse_apply_kernel<<<blocks_for(n * 32, 256), 256, 0, s>>>(inv, n, g, u);
    return cudaGetLastError();
}

cudaError_t launch_d2f(const double *x, float *y, int64_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    note_launches(1);
    d2f_kernel<<<blocks_for(n, 256), 256, 0, s>>>(x, y, n);
    return cudaGetLastError();
}
cudaError_t launch_f2d(const float *x, double *y, int64_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    note_launches(1);
    f2d_kernel<<<blocks_for(n, 256), 256, 0, s>>>(x, y, n);
    return cudaGetLastError();
}
template <class T>
cudaError_t launch_fill(T *x, T v, int64_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    note_launches(1);
    fill_kernel<T><<<blocks_for(n, 256), 256, 0, s>>>(x, v, n);
    return cudaGetLastError();
}
cudaError_t launch_axpby(double a, const double *x, double b, double *y, int64_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    note_launches(1);
    axpby_kernel<<<blocks_for(n, 256), 256, 0, s>>>(a, x, b, y, n);
    return cudaGetLastError();
}

int krylov_partial_blocks() { return KRYLOV_BLOCKS; }

template <int NVB>
static void dots_nvb(const double *V, int nv, int64_t ld, const double *w, int64_t n, double *partials,
                     cudaStream_t s) {
    note_launches(1);
    dim3 grid(KRYLOV_BLOCKS, (nv + 15) / 16);
    dots_kernel<NVB><<<grid, KRYLOV_THREADS, 0, s>>>(V, nv, ld, w, n, partials);
}

cudaError_t launch_dots(const double *V, int nv, int64_t ld, const double *w, int64_t n, double *partials,
                        cudaStream_t s) {
    if (nv < 1 || nv > MAXV) return cudaErrorInvalidValue;
    if (nv <= 1) dots_nvb<1>(V, nv, ld, w, n, partials, s);
    else if (nv <= 2) dots_nvb<2>(V, nv, ld, w, n, partials, s);
    else if (nv <= 4) dots_nvb<4>(V, nv, ld, w, n, partials, s);
    else if (nv <= 8) dots_nvb<8>(V, nv, ld, w, n, partials, s);
    else dots_nvb<16>(V, nv, ld, w, n, partials, s);
    return cudaGetLastError();
}

template <int NVB, int MODE>
static void upd(const double *V, int nv, int64_t ld, double *w, int64_t n, const double *h, double *partials,
                cudaStream_t s) {
    note_launches(1);
    update_dots_kernel<NVB, MODE><<<KRYLOV_BLOCKS, KRYLOV_THREADS, 0, s>>>(V, nv, ld, w, n, h, partials);
}

// mode 1: w -= V h and partial dots <V_i, w>; mode 2: w -= V h and partial <w, w>
cudaError_t launch_update_dots(const double *V, int nv, int64_t ld, double *w, int64_t n, const double *h,
                               double *partials, int mode, cudaStream_t s) {
    if (nv < 1 || nv > MAXV) return cudaErrorInvalidValue;
    if (mode == 2) {
        upd<1, 2>(V, nv, ld, w, n, h, partials, s);
    } else if (nv <= 4) {
        upd<4, 1>(V, nv, ld, w, n, h, partials, s);
    } else if (nv <= 8) {
        upd<8, 1>(V, nv, ld, w, n, h, partials, s);
    } else if (nv <= 16) {
        upd<16, 1>(V, nv, ld, w, n, h, partials, s);
    } else {
        upd<1, 0>(V, nv, ld, w, n, h, partials, s);
        return launch_dots(V, nv, ld, w, n, partials, s);
    }
    return cudaGetLastError();
}

cudaError_t launch_reduce_partials(const double *partials, int nv, double *out, int accumulate,
                                   cudaStream_t s) {
    note_launches(1);
    reduce_partials_kernel<<<nv, 32, 0, s>>>(partials, nv, KRYLOV_BLOCKS, out, accumulate);
    return cudaGetLastError();
}
cudaError_t launch_givens(double *small, int j, int restart, double *, cudaStream_t s) {
    note_launches(1);
    givens_kernel<<<1, 1, 0, s>>>(small, j, restart);
    return cudaGetLastError();
}
cudaError_t launch_scale_next(const double *w, double *v, int64_t n, const double *small, int,
                              int restart, cudaStream_t s) {
    SmallLayout Ly{restart};
    note_launches(1);
    scale_next_kernel<<<blocks_for(n, 256), 256, 0, s>>>(w, v, n, small, Ly.hn());
    return cudaGetLastError();
}
cudaError_t launch_init_cycle(const double *r, double *v0, int64_t n, double *small, int restart,
                              cudaStream_t s) {
    int64_t m = n > restart + 1 ? n : restart + 1;
    note_launches(1);
    init_cycle_kernel<<<blocks_for(m, 256), 256, 0, s>>>(r, v0, n, small, restart);
    return cudaGetLastError();
}
cudaError_t launch_solve_update(double *small, int m, int restart, const double *Z, int64_t ld, double *x,
                                int64_t n, cudaStream_t s) {
    SmallLayout Ly{restart};
    note_launches(1);
    backsolve_kernel<<<1, 1, 0, s>>>(small, m, restart);
    note_launches(1);
    update_x_kernel<<<blocks_for(n, 256), 256, 0, s>>>(Z, m, ld, small, Ly.y(), x, n);
    return cudaGetLastError();
}
cudaError_t launch_uzawa_rhs(const DevLevel &L, int k, const double *F, const double *p, double *g,
                             cudaStream_t s) {
    int dpf = dpf_of(L.dim, k);
    int64_t n = L.n_int * dpf;
    if (n == 0) return cudaSuccess;
    note_launches(1);
    uzawa_rhs_kernel<<<blocks_for(n, 256), 256, 0, s>>>(L.n_int, dpf, L.dim + 1, L.facet_adj.p, L.cell_d.p, F, p,
                                                         g);
    return cudaGetLastError();
}
__global__ void __launch_bounds__(KRYLOV_THREADS)
sum_kernel(const double *__restrict__ x, int64_t n, double *__restrict__ partials) {
    double acc[1] = {0.0};
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        acc[0] += x[e];
    block_reduce_store<1>(acc, 1, partials);
}

cudaError_t launch_sum(const double *x, int64_t n, double *partials, cudaStream_t s) {
    note_launches(1);
    sum_kernel<<<KRYLOV_BLOCKS, KRYLOV_THREADS, 0, s>>>(x, n, partials);
    return cudaGetLastError();
}

cudaError_t launch_uzawa_update(const DevLevel &L, int k, const double *u, double *p, double gamma, double nu,
                                const double *nu_cell, const double *bflux, double *partials, cudaStream_t s) {
    note_launches(1);
    uzawa_update_kernel<<<KRYLOV_BLOCKS, KRYLOV_THREADS, 0, s>>>(L.nc, dpf_of(L.dim, k), L.dim + 1, L.cell_int.p,
                                                                 L.cell_d.p,
                                                                 L.cell_area.p, u, p, gamma, nu, nu_cell, bflux,
                                                                 partials);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- transposed apply
// y = A^T x, pull style: the row of unknown (facet i, component d) in A^T is its column in the
// element matrices of its two cells, A_K[(f2, d2), q] with q = lf dpf + d; with the row-block
// layout that entry sits at (f2 n_loc + q) dpf + d2
template <int DPF>
__global__ void apply_t_kernel(int64_t n_int, const int *__restrict__ facet_adj, const int *__restrict__ cell_int,
                               const double *__restrict__ A, const double *__restrict__ x, double *__restrict__ y) {
    constexpr int NLOC = 3 * DPF;
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n_int * DPF) return;
    const int64_t i = idx / DPF;
    const int d = (int)(idx - i * DPF);
    double acc = 0.0;
    for (int q2 = 0; q2 < 2; ++q2) {
        const int adj = facet_adj[2 * i + q2];
        if (adj < 0) continue;
        const int c = adj >> 2, lf = adj & 3;
        const int q = lf * DPF + d;
        const double *Ac = A + (size_t)c * NLOC * NLOC;
        for (int f2 = 0; f2 < 3; ++f2) {
            const int j = cell_int[3 * c + f2];
            if (j < 0) continue;
            const double *Ar = Ac + ((size_t)f2 * NLOC + q) * DPF;
            for (int d2 = 0; d2 < DPF; ++d2) acc += Ar[d2] * x[(size_t)j * DPF + d2];
        }
    }
    y[idx] = acc;
}

cudaError_t launch_apply_t(const DevLevel &L, const DevOperator &op, const double *x, double *y, cudaStream_t s) {
    const int64_t n = L.n_int * op.dpf;
    if (n == 0) return cudaSuccess;
    note_launches(1);
    switch (op.dpf) {
#define HDG_APT(D) \
    case D: apply_t_kernel<D><<<blocks_for(n, 256), 256, 0, s>>>(L.n_int, L.facet_adj.p, L.cell_int.p, op.A.p, x, y); break;
    HDG_APT(2) HDG_APT(4) HDG_APT(6) HDG_APT(8) HDG_APT(10)
#undef HDG_APT
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- inhomogeneous Dirichlet data
// F_i -= sum over the facet's cells of A_K[row i, boundary columns] u_D (pull style, like the
// apply: each interior facet row reads its two cells' row blocks at the boundary facets' columns)
template <int DPF, int NFC>
__global__ void dirichlet_load_kernel(int64_t n_int, const int *__restrict__ facet_adj,
                                      const int *__restrict__ cell_bnd, const double *__restrict__ A,
                                      const double *__restrict__ xD, double *__restrict__ F) {
    constexpr int NLOC = NFC * DPF;
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n_int * DPF) return;
    const int64_t i = idx / DPF;
    const int d = (int)(idx - i * DPF);
    double acc = 0.0;
    for (int q = 0; q < 2; ++q) {
        const int adj = facet_adj[2 * i + q];
        if (adj < 0) continue;
        const int c = adj >> 2, lf = adj & 3;
        const double *Ac = A + (size_t)c * NLOC * NLOC + lf * NLOC * DPF + d;
        for (int f2 = 0; f2 < NFC; ++f2) {
            const int b = cell_bnd[NFC * c + f2];
            if (b < 0) continue;
            for (int d2 = 0; d2 < DPF; ++d2) acc += Ac[(f2 * DPF + d2) * DPF] * xD[(size_t)b * DPF + d2];
        }
    }
    F[idx] -= acc;
}

// per cell, the flux of the Dirichlet data through its boundary facets: sum of d_f (normal moment 0)
__global__ void boundary_flux_kernel(int64_t nc, int dpf, int nfc, const int *__restrict__ cell_bnd,
                                     const double *__restrict__ cell_d, const double *__restrict__ xD,
                                     double *__restrict__ bflux) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= nc) return;
    double s = 0.0;
    for (int f = 0; f < nfc; ++f) {
        const int b = cell_bnd[nfc * c + f];
        if (b >= 0) s += cell_d[nfc * c + f] * xD[(size_t)b * dpf];
    }
    bflux[c] = s;
}

cudaError_t launch_dirichlet_load(const DevLevel &L, const DevOperator &op, const double *xD, double *F,
                                  cudaStream_t s) {
    const int64_t n = L.n_int * op.dpf;
    if (n == 0) return cudaSuccess;
    note_launches(1);
    if (L.dim == 3) {
        switch (op.dpf) {
#define HDG_DIR3(D) \
        case D: dirichlet_load_kernel<D, 4><<<blocks_for(n, 256), 256, 0, s>>>(L.n_int, L.facet_adj.p, L.cell_bnd.p, op.A.p, xD, F); break;
        HDG_DIR3(3) HDG_DIR3(9) HDG_DIR3(18) HDG_DIR3(30)
#undef HDG_DIR3
        default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    switch (op.dpf) {
#define HDG_DIR(D) \
    case D: dirichlet_load_kernel<D, 3><<<blocks_for(n, 256), 256, 0, s>>>(L.n_int, L.facet_adj.p, L.cell_bnd.p, op.A.p, xD, F); break;
    HDG_DIR(2) HDG_DIR(4) HDG_DIR(6) HDG_DIR(8) HDG_DIR(10)
#undef HDG_DIR
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_boundary_flux(const DevLevel &L, int dpf, const double *xD, double *bflux, cudaStream_t s) {
    if (L.nc == 0) return cudaSuccess;
    note_launches(1);
    boundary_flux_kernel<<<blocks_for(L.nc, 256), 256, 0, s>>>(L.nc, dpf, L.dim + 1, L.cell_bnd.p, L.cell_d.p, xD,
                                                                bflux);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- damped block Jacobi (eq. bjac)
// Step one: every patch solves against the same residual r = g - A u (one block per patch,
// patch row t on thread t): D[p np_max + t] = sum_j (A_P^-1)_tj r_{P,j}.
template <class T, int DPF>
__global__ void jacobi_patch_kernel(int n_patches, int pf_max, int np_max, const int *__restrict__ patch_nf,
                                    const int *__restrict__ patch_facets, const T *__restrict__ Pinv,
                                    const T *__restrict__ r, T *__restrict__ D) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T *rs = reinterpret_cast<T *>(smraw);   // np_max
    const int p = blockIdx.x;
    if (p >= n_patches) return;
    const int np = patch_nf[p] * DPF;
    for (int t = threadIdx.x; t < np; t += blockDim.x)
        rs[t] = r[(size_t)patch_facets[(size_t)p * pf_max + t / DPF] * DPF + t % DPF];
    __syncthreads();
    const T *Pi = Pinv + (size_t)p * np_max * np_max;
    for (int t = threadIdx.x; t < np; t += blockDim.x) {
        T acc = 0;
        for (int j = 0; j < np; ++j) acc += Pi[(size_t)j * np_max + t] * rs[j];
        D[(size_t)p * np_max + t] = acc;
    }
}

// Step two: each interior facet lies in the patches of its two vertices; its unknowns add
// the two corrections in a fixed order, scaled by the damping s:
// u_F += s (D[slot_a] + D[slot_b]), slot = patch p x pf_max + position of F in the patch
template <class T, int DPF>
__global__ void jacobi_gather_kernel(int64_t n_int, const int *__restrict__ facet_slot, T s,
                                     const T *__restrict__ D, T *__restrict__ u) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n_int * DPF) return;
    const int64_t F = idx / DPF;
    const int d = (int)(idx - F * DPF);
    const int a = facet_slot[2 * F], b = facet_slot[2 * F + 1];
    T acc = 0;
    if (a >= 0) acc += D[(size_t)a * DPF + d];
    if (b >= 0) acc += D[(size_t)b * DPF + d];
    u[idx] += s * acc;
}

template <class T, int DPF>
cudaError_t jacobi_launch(const DevLevel &L, const DevOperator &op, const T *Pinv, const T *r, T *D, T damping,
                          T *u, cudaStream_t s) {
    if (L.n_patches > 0) {
        int nt = ((op.np_max + 31) / 32) * 32;
        nt = nt > 256 ? 256 : nt;
        note_launches(1);
        jacobi_patch_kernel<T, DPF><<<L.n_patches, nt, sizeof(T) * op.np_max, s>>>(
            L.n_patches, L.pf_max, op.np_max, L.patch_nf.p, L.patch_facets.p, Pinv, r, D);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const int64_t n = L.n_int * DPF;
    if (n == 0) return cudaSuccess;
    note_launches(1);
    jacobi_gather_kernel<T, DPF><<<blocks_for(n, 256), 256, 0, s>>>(L.n_int, L.facet_slot.p, damping, D, u);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_jacobi_update(const DevLevel &L, const DevOperator &op, const T *Pinv, const T *r, T *D,
                                 double damping, T *u, cudaStream_t s) {
    switch (op.dpf) {
    case 2: return jacobi_launch<T, 2>(L, op, Pinv, r, D, (T)damping, u, s);
    case 4: return jacobi_launch<T, 4>(L, op, Pinv, r, D, (T)damping, u, s);
    case 6: return jacobi_launch<T, 6>(L, op, Pinv, r, D, (T)damping, u, s);
    case 8: return jacobi_launch<T, 8>(L, op, Pinv, r, D, (T)damping, u, s);
    case 10: return jacobi_launch<T, 10>(L, op, Pinv, r, D, (T)damping, u, s);
    default: return cudaErrorInvalidValue;
    }
}

// explicit instantiations
template cudaError_t launch_jacobi_update<double>(const DevLevel &, const DevOperator &, const double *,
                                                  const double *, double *, double, double *, cudaStream_t);
template cudaError_t launch_jacobi_update<float>(const DevLevel &, const DevOperator &, const float *,
                                                 const float *, float *, double, float *, cudaStream_t);
template cudaError_t launch_apply<double>(const DevLevel &, const DevOperator &, const double *,
                                          const double *, const double *, double *, cudaStream_t);
template cudaError_t launch_apply<float>(const DevLevel &, const DevOperator &, const float *, const float *,
                                         const float *, float *, cudaStream_t);
template cudaError_t launch_gs_colour<double>(const DevLevel &, const DevOperator &, const double *,
                                              const double *, int, const double *, double *, cudaStream_t);
template cudaError_t launch_gs_colour<float>(const DevLevel &, const DevOperator &, const float *,
                                             const float *, int, const float *, float *, cudaStream_t);
template cudaError_t launch_prolong_add<double>(const DevLevel &, const DevLevel &, const double *,
                                                const double *, const double *, double *, double *,
                                                cudaStream_t);
template cudaError_t launch_prolong_add<float>(const DevLevel &, const DevLevel &, const float *,
                                               const float *, const float *, float *, float *, cudaStream_t);
template cudaError_t launch_restrict<double>(const DevLevel &, const DevLevel &, const double *,
                                             const double *, const double *, double *, double *, double *,
                                             cudaStream_t);
template cudaError_t launch_restrict<float>(const DevLevel &, const DevLevel &, const float *, const float *,
                                            const float *, float *, float *, float *, cudaStream_t);
template cudaError_t launch_hp_restrict<double>(int, int64_t, const double *, double *, cudaStream_t);
template cudaError_t launch_hp_restrict<float>(int, int64_t, const float *, float *, cudaStream_t);
template cudaError_t launch_hp_prolong_add<double>(int, int64_t, const double *, double *, cudaStream_t);
template cudaError_t launch_hp_prolong_add<float>(int, int64_t, const float *, float *, cudaStream_t);
template cudaError_t launch_fill<double>(double *, double, int64_t, cudaStream_t);
template cudaError_t launch_fill<float>(float *, float, int64_t, cudaStream_t);

} // namespace hdg
