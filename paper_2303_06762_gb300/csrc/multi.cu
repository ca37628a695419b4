// Multi-right-hand-side (batched) kernels: the hot path for R systems that
// share one condensed operator (several loads on one mesh).
//
// A multi-vector holds R columns interleaved by row, X[row][R] (the column
// index fastest), R a power of two <= 64.  The R consecutive threads of one
// row read the same element-matrix or patch-inverse entry (one broadcast
// transaction) and R consecutive vector values, so every matrix byte fetched
// from HBM serves all R right-hand sides: the operator apply, the block
// Gauss-Seidel sweep and the transfers of Algorithms 1 and 2 become products
// of the stored local matrices with R-column blocks.  Krylov reductions keep
// one accumulator per (vector, column) and reduce each column separately, so
// the R flexible GMRES iterations of hdg_solve_multi stay independent.  The
// order-k sweep's tile (rows per thread, threads per block) is a launch
// parameter chosen by the host autotuner; the 16-bit precisions run that sweep
// on tensor cores instead (multi_tc.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "hdg_internal.h"

namespace hdg {
namespace {

constexpr int MT = 256;          // threads per block of the element-wise kernels
constexpr int MAXVM = 33;        // Krylov basis vectors (restart <= 32)

unsigned nblk(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// ---------------------------------------------------------------- operator apply
// y = A x (or y = g - A x) for R = 2^lgR columns, pull style per facet row.  A
// thread owns RB consecutive rows of one facet and one column: every x value it
// loads feeds RB products.
template <class T, int DPF, int RB>
__global__ void __launch_bounds__(MT)
apply_m_kernel(int64_t n_int, int lgR, const int *__restrict__ facet_adj, const int *__restrict__ cell_int,
               const T *__restrict__ A, const T *__restrict__ x, const T *__restrict__ g, T *__restrict__ y) {
    constexpr int NLOC = 3 * DPF;
    const int R = 1 << lgR;
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= (n_int * (DPF / RB)) << lgR) return;
    const int64_t rb = idx >> lgR;
    const int r = (int)(idx & (R - 1));
    const int64_t i = rb / (DPF / RB);
    const int d0 = (int)(rb - i * (DPF / RB)) * RB;
    T acc[RB];
#pragma unroll
    for (int b = 0; b < RB; ++b) acc[b] = 0;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int adj = facet_adj[2 * i + q];
        if (adj < 0) continue;
        const int c = adj >> 2, lf = adj & 3;
        const T *Ac = A + (size_t)c * NLOC * NLOC + lf * NLOC * DPF + d0;
#pragma unroll
        for (int f2 = 0; f2 < 3; ++f2) {
            const int j = cell_int[3 * c + f2];
            if (j < 0) continue;
            const T *xs = x + ((size_t)j * DPF << lgR) + r;
#pragma unroll
            for (int d2 = 0; d2 < DPF; ++d2) {
                const T xv = xs[(size_t)d2 << lgR];
                const T *a = Ac + (f2 * DPF + d2) * DPF;
#pragma unroll
                for (int b = 0; b < RB; ++b) acc[b] += a[b] * xv;
            }
        }
    }
    const size_t o = (((size_t)i * DPF + d0) << lgR) + r;
#pragma unroll
    for (int b = 0; b < RB; ++b) {
        const size_t e = o + ((size_t)b << lgR);
        y[e] = g ? g[e] - acc[b] : acc[b];
    }
}

// y = A x (or g - A x) in double-FP32 arithmetic: A = A_hi + A_lo (two FP32 words),
// each x value split the same way, products formed exactly (FMA residual) plus
// the two cross terms, sums kept as unevaluated FP32 pairs (two-sum).  The result
// carries about 44 significant bits at the FP32 issue rate, where GB300's FP64
// units would bound the same apply at a few percent of that rate.
__device__ __forceinline__ void df_add(float &sh, float &sl, float p, float c) {
    const float t = sh + p;
    const float z = t - sh;
    const float err = (sh - (t - z)) + (p - z);
    sh = t;
    sl += err + c;
}

template <int DPF, int RB>
__global__ void __launch_bounds__(MT)
apply_df_m_kernel(int64_t n_int, int lgR, const int *__restrict__ facet_adj, const int *__restrict__ cell_int,
                  const float *__restrict__ Ahi, const float *__restrict__ Alo, const float2 *__restrict__ xp,
                  const double *__restrict__ g, double *__restrict__ y) {
    constexpr int NLOC = 3 * DPF;
    const int R = 1 << lgR;
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= (n_int * (DPF / RB)) << lgR) return;
    const int64_t rb = idx >> lgR;
    const int r = (int)(idx & (R - 1));
    const int64_t i = rb / (DPF / RB);
    const int d0 = (int)(rb - i * (DPF / RB)) * RB;
    float sh[RB], sl[RB];
#pragma unroll
    for (int b = 0; b < RB; ++b) sh[b] = sl[b] = 0.0f;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int adj = facet_adj[2 * i + q];
        if (adj < 0) continue;
        const int c = adj >> 2, lf = adj & 3;
        const size_t base = (size_t)c * NLOC * NLOC + lf * NLOC * DPF + d0;
#pragma unroll
        for (int f2 = 0; f2 < 3; ++f2) {
            const int j = cell_int[3 * c + f2];
            if (j < 0) continue;
            const float2 *xs = xp + ((size_t)j * DPF << lgR) + r;
#pragma unroll
            for (int d2 = 0; d2 < DPF; ++d2) {
                const float2 xv = xs[(size_t)d2 << lgR];      // (hi, lo) of x
                const size_t o = base + (size_t)(f2 * DPF + d2) * DPF;
#pragma unroll
                for (int b = 0; b < RB; ++b) {
                    const float ah = Ahi[o + b], al = Alo[o + b];
                    const float p = ah * xv.x;
                    const float e = fmaf(ah, xv.x, -p);
                    const float cr = fmaf(ah, xv.y, fmaf(al, xv.x, e));
                    df_add(sh[b], sl[b], p, cr);
                }
            }
        }
    }
    const size_t o = (((size_t)i * DPF + d0) << lgR) + r;
#pragma unroll
    for (int b = 0; b < RB; ++b) {
        const size_t e = o + ((size_t)b << lgR);
        const double v = (double)sh[b] + (double)sl[b];
        y[e] = g ? g[e] - v : v;
    }
}

// x -> (hi, lo) FP32 pairs, hi = fl32(x), lo = fl32(x - hi)
__global__ void split_x_kernel(const double *__restrict__ x, float2 *__restrict__ xp, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = x[i];
    const float h = (float)v;
    xp[i] = make_float2(h, (float)(v - (double)h));
}

// lo = (float)(A - (double)hi): the FP32 remainder of the FP32 copy hi of A
__global__ void split_lo_kernel(const double *__restrict__ A, const float *__restrict__ hi, float *__restrict__ lo,
                                int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) lo[i] = (float)(A[i] - (double)hi[i]);
}

// ---------------------------------------------------------------- block Gauss-Seidel, one colour
template <class T>
struct Pair;
template <>
struct Pair<float> {
    using type = float2;
};
template <>
struct Pair<double> {
    using type = double2;
};

// u_s += A_ss^{-1} (g - A u)_s for every patch s of the colour, R = 2^lgR columns at
// once.  The patch's index tables, the element-matrix rows of its facets and its
// block inverse are first staged in shared memory with independent, coalesced
// pair-wide loads; the residual and the block solve then read only shared memory
// (one broadcast entry per R columns).  A thread owns RB rows of one column.
// EXT: the closed form u_s = A_ss^{-1} (g_s - A_sE u_E) (E = each star cell's facet
// opposite the patch vertex, patch_cext; equal to the update above because Pinv inverts
// the assembled A_ss): the rows' coupling blocks with E and the unknowns on E only.  With
// swQ (FP32) the augmented-Lagrangian term is split off, A_ss^{-1} (g_s - A0_sE u_E) - Q z
// with z the star cells' outside fluxes, so that no O(gamma) value meets the FP32 inverse.
template <class T, int DPF, int RB, bool EXT>
__global__ void __launch_bounds__(MT)
gs_m_kernel(int p0, int p1, int pf_max, int pc_max, int np_max, int lgR, const int *__restrict__ patch_nf,
            const int *__restrict__ patch_facets, const int *__restrict__ patch_nc,
            const int *__restrict__ patch_cells, const int *__restrict__ slot_src,
            const int *__restrict__ cell_int, const int *__restrict__ patch_cext, const float *__restrict__ swQ,
            const float *__restrict__ swA00, const double *__restrict__ cell_d, const T *__restrict__ A,
            const T *__restrict__ Pinv, const T *__restrict__ g, T *__restrict__ u) {
    using T2 = typename Pair<T>::type;
    constexpr int NLOC = 3 * DPF;
    constexpr int NX = EXT ? DPF : NLOC;                        // columns read per row, unknowns per cell
    const int R = 1 << lgR;
    extern __shared__ __align__(16) unsigned char smraw[];
    T *xs = reinterpret_cast<T *>(smraw);                       // pc_max * NX * R
    T *rs = xs + ((size_t)pc_max * NX << lgR);                  // np_max * R
    T *As = rs + ((size_t)np_max << lgR);                       // pf_max * 2 * NX * DPF
    T *Ps = As + (size_t)pf_max * 2 * NX * DPF;                 // np_max * np_max
    int *jt = reinterpret_cast<int *>(Ps + (size_t)np_max * np_max);   // pc_max * 3
    int *rowF = jt + pc_max * 3;                                // pf_max
    int *rowA = rowF + pf_max;                                  // pf_max * 2
    int *rowS = rowA + pf_max * 2;                              // pf_max * 2
    T *zs = reinterpret_cast<T *>(jt + ((pc_max * 3 + pf_max * 5 + 3) & ~3));   // pc_max * R (split form)
    const int p = p0 + blockIdx.x;
    if (p >= p1) return;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int nf = patch_nf[p], ncell = patch_nc[p], np = nf * DPF;
    const bool split = EXT && swQ;
    if constexpr (EXT) {
        for (int i = tid; i < ncell; i += nt)
            jt[i] = cell_int[3 * patch_cells[(size_t)p * pc_max + i] + patch_cext[(size_t)p * pc_max + i]];
    } else {
        for (int i = tid; i < ncell * 3; i += nt) {
            const int c = patch_cells[(size_t)p * pc_max + i / 3];
            jt[i] = cell_int[3 * c + i % 3];
        }
    }
    for (int js = tid; js < nf; js += nt) {
        rowF[js] = patch_facets[(size_t)p * pf_max + js];
        for (int q = 0; q < 2; ++q) {
            const int src = slot_src[((size_t)p * pf_max + js) * 2 + q];
            const int si = src >> 2, lf = src & 3;
            const int c = patch_cells[(size_t)p * pc_max + si];
            rowA[2 * js + q] = c * NLOC * NLOC + lf * NLOC * DPF +
                               (EXT ? patch_cext[(size_t)p * pc_max + si] * DPF * DPF : 0);
            rowS[2 * js + q] = si;
        }
    }
    {   // block inverse, whole np_max x np_max block (contiguous)
        const T2 *src = reinterpret_cast<const T2 *>(Pinv + (size_t)p * np_max * np_max);
        T2 *dst = reinterpret_cast<T2 *>(Ps);
        const int n2 = np_max * np_max / 2;
#pragma unroll 4
        for (int i = tid; i < n2; i += nt) dst[i] = src[i];
    }
    __syncthreads();
    {   // rows (lf, 0..DPF) of every column read (all, or the outside facet's) of the two
        // cells of each patch facet
        constexpr int U = DPF / 2;              // pairs per column
        const int n2 = nf * 2 * NX * U;
#pragma unroll 4
        for (int i = tid; i < n2; i += nt) {
            const int h = i % U, col = (i / U) % NX, jq = i / (U * NX);
            const T2 *src = reinterpret_cast<const T2 *>(A + rowA[jq] + col * DPF) + h;
            T2 v = *src;
            if (split && h == 0 && col == 0) v.x = (T)swA00[(size_t)p * pf_max * 2 + jq];   // AL-free (0, 0)
            reinterpret_cast<T2 *>(As)[i] = v;
        }
    }
#pragma unroll 4
    for (int t = tid; t < (ncell * NX) << lgR; t += nt) {
        const int r = t & (R - 1), sl = t >> lgR, si = sl / NX, l = sl - si * NX;
        const int j = EXT ? jt[si] : jt[si * 3 + l / DPF];
        const T x = j >= 0 ? u[(((size_t)j * DPF + l % DPF) << lgR) + r] : T(0);
        xs[t] = x;
        if (split && l == 0) {
            const int c = patch_cells[(size_t)p * pc_max + si];
            zs[(si << lgR) + r] = (T)cell_d[3 * (size_t)c + patch_cext[(size_t)p * pc_max + si]] * x;
        }
    }
    __syncthreads();
    const int nrb = np / RB;
    for (int t = tid; t < nrb << lgR; t += nt) {
        const int r = t & (R - 1), row0 = (t >> lgR) * RB, js = row0 / DPF, d0 = row0 - js * DPF;
        const int F = rowF[js];
        T acc[RB];
#pragma unroll
        for (int b = 0; b < RB; ++b) acc[b] = g[(((size_t)F * DPF + d0 + b) << lgR) + r];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const T *Ac = As + (size_t)(2 * js + q) * NX * DPF + d0;
            const T *xc = xs + ((size_t)rowS[2 * js + q] * NX << lgR) + r;
#pragma unroll
            for (int col = 0; col < NX; ++col) {
                const T xv = xc[col << lgR];
                const T *a = Ac + col * DPF;
#pragma unroll
                for (int b = 0; b < RB; ++b) acc[b] -= a[b] * xv;
            }
        }
#pragma unroll
        for (int b = 0; b < RB; ++b) rs[((row0 + b) << lgR) + r] = acc[b];
    }
    __syncthreads();
    for (int t = tid; t < nrb << lgR; t += nt) {
        const int r = t & (R - 1), row0 = (t >> lgR) * RB;
        T acc[RB];
#pragma unroll
        for (int b = 0; b < RB; ++b) acc[b] = 0;
#pragma unroll 4
        for (int j = 0; j < np; ++j) {
            const T xv = rs[(j << lgR) + r];
            const T *pj = Ps + j * np_max + row0;
#pragma unroll
            for (int b = 0; b < RB; ++b) acc[b] += pj[b] * xv;
        }
        if (split)
            for (int si = 0; si < ncell; ++si) {
                const T z = zs[(si << lgR) + r];
                const float *qc = swQ + ((size_t)p * pc_max + si) * np_max + row0;
#pragma unroll
                for (int b = 0; b < RB; ++b) acc[b] -= (T)qc[b] * z;
            }
        const int js = row0 / DPF, d0 = row0 - js * DPF;
        const size_t o = (((size_t)rowF[js] * DPF + d0) << lgR) + r;
#pragma unroll
        for (int b = 0; b < RB; ++b) {
            if constexpr (EXT) u[o + ((size_t)b << lgR)] = acc[b];
            else u[o + ((size_t)b << lgR)] += acc[b];
        }
    }
}

// ---------------------------------------------------------------- order-k <-> lowest order
template <class T>
__global__ void hp_restrict_m_kernel(int k, int64_t n_int, int R, const T *__restrict__ r, T *__restrict__ r0) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n_int * R) return;
    const int64_t i = idx / R;
    const int c = (int)(idx - i * R);
    const int dpf = 2 * (k + 1);
    r0[(2 * i) * R + c] = r[(i * dpf) * R + c];
    r0[(2 * i + 1) * R + c] = r[(i * dpf + k + 1) * R + c];
}

template <class T>
__global__ void hp_prolong_m_kernel(int k, int64_t n_int, int R, const T *__restrict__ d0, T *__restrict__ u) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n_int * R) return;
    const int64_t i = idx / R;
    const int c = (int)(idx - i * R);
    const int dpf = 2 * (k + 1);
    u[(i * dpf) * R + c] += d0[(2 * i) * R + c];
    u[(i * dpf + k + 1) * R + c] += d0[(2 * i + 1) * R + c];
}

// ---------------------------------------------------------------- lowest-order transfers
template <class T>
__global__ void prolong_B_m_kernel(int64_t nB, int R, const int *__restrict__ fineB,
                                   const int *__restrict__ fineB_src, const int *__restrict__ ccell_int,
                                   const T *__restrict__ W, const T *__restrict__ uc, T *__restrict__ tmp,
                                   T *__restrict__ uf) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= nB * R) return;
    const int64_t b = idx / R;
    const int r = (int)(idx - b * R);
    T v0 = 0, v1 = 0;
    for (int q = 0; q < 2; ++q) {
        const int src = fineB_src[2 * b + q];
        const int P = src >> 4, s = src & 15;
        const T *Wk = W + (size_t)P * 72;
        for (int fp = 0; fp < 3; ++fp) {
            const int j = ccell_int[3 * P + fp];
            if (j < 0) continue;
            for (int cq = 0; cq < 2; ++cq) {
                const T u = uc[(2 * (size_t)j + cq) * R + r];
                v0 += Wk[(2 * s) * 6 + 2 * fp + cq] * u;
                v1 += Wk[(2 * s + 1) * 6 + 2 * fp + cq] * u;
            }
        }
    }
    const size_t i = fineB[b];
    tmp[(2 * i) * R + r] = v0;
    tmp[(2 * i + 1) * R + r] = v1;
    uf[(2 * i) * R + r] += v0;
    uf[(2 * i + 1) * R + r] += v1;
}

template <class T>
__global__ void prolong_T_m_kernel(int64_t ncc, int R, const int *__restrict__ slots, const T *__restrict__ H,
                                   const T *__restrict__ tmp, T *__restrict__ uf) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= ncc * R) return;
    const int64_t P = idx / R;
    const int r = (int)(idx - P * R);
    T b[12];
    for (int s = 0; s < 6; ++s) {
        const int i = slots[9 * P + s];
        b[2 * s] = i >= 0 ? tmp[(2 * (size_t)i) * R + r] : T(0);
        b[2 * s + 1] = i >= 0 ? tmp[(2 * (size_t)i + 1) * R + r] : T(0);
    }
    const T *Hk = H + (size_t)P * 72;
    for (int t = 0; t < 6; ++t) {
        T acc = 0;
        for (int c = 0; c < 12; ++c) acc += Hk[t * 12 + c] * b[c];
        const size_t i = slots[9 * P + 6 + t / 2];
        uf[(2 * i + (t & 1)) * R + r] += acc;
    }
}

template <class T>
__global__ void restrict_T_m_kernel(int64_t ncc, int R, const int *__restrict__ slots, const T *__restrict__ H,
                                    const T *__restrict__ rf, T *__restrict__ t1) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= ncc * R) return;
    const int64_t P = idx / R;
    const int r = (int)(idx - P * R);
    T rT[6];
    for (int t = 0; t < 6; ++t) rT[t] = rf[(2 * (size_t)slots[9 * P + 6 + t / 2] + (t & 1)) * R + r];
    const T *Hk = H + (size_t)P * 72;
    for (int c = 0; c < 12; ++c) {
        T acc = 0;
        for (int t = 0; t < 6; ++t) acc += Hk[t * 12 + c] * rT[t];
        t1[(12 * P + c) * R + r] = acc;
    }
}

template <class T>
__global__ void restrict_B_m_kernel(int64_t ncc, int R, const int *__restrict__ slots, const int *__restrict__ nbr,
                                    const T *__restrict__ W, const T *__restrict__ rf, const T *__restrict__ t1,
                                    T *__restrict__ t2) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= ncc * R) return;
    const int64_t P = idx / R;
    const int r = (int)(idx - P * R);
    T z[12];
    for (int s = 0; s < 6; ++s) {
        const int i = slots[9 * P + s];
        if (i < 0) {
            z[2 * s] = z[2 * s + 1] = 0;
            continue;
        }
        const int nb = nbr[6 * P + s];
        const int64_t Q = nb >> 4;
        const int s2 = nb & 15;
        for (int c = 0; c < 2; ++c)
            z[2 * s + c] = rf[(2 * (size_t)i + c) * R + r] + t1[(12 * P + 2 * s + c) * R + r] +
                           t1[(12 * Q + 2 * s2 + c) * R + r];
    }
    const T *Wk = W + (size_t)P * 72;
    for (int col = 0; col < 6; ++col) {
        T acc = 0;
        for (int row = 0; row < 12; ++row) acc += Wk[row * 6 + col] * z[row];
        t2[(6 * P + col) * R + r] = acc;
    }
}

template <class T>
__global__ void restrict_C_m_kernel(int64_t n_int_c, int R, const int *__restrict__ facet_adj_c,
                                    const T *__restrict__ t2, T *__restrict__ rc) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n_int_c * R) return;
    const int64_t G = idx / R;
    const int r = (int)(idx - G * R);
    T a0 = 0, a1 = 0;
    for (int q = 0; q < 2; ++q) {
        const int adj = facet_adj_c[2 * G + q];
        const int64_t K = adj >> 2;
        const int lf = adj & 3;
        a0 += t2[(6 * K + 2 * lf) * R + r];
        a1 += t2[(6 * K + 2 * lf + 1) * R + r];
    }
    rc[(2 * G) * R + r] = a0;
    rc[(2 * G + 1) * R + r] = a1;
}

// u = inv g for R columns (coarsest level, FP64 inverse); g, u of type T
template <class T>
__global__ void coarse_m_kernel(const double *__restrict__ inv, int64_t n, int R, const T *__restrict__ g,
                                T *__restrict__ u) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n * R) return;
    const int64_t row = idx / R;
    const int r = (int)(idx - row * R);
    double acc = 0.0;
    const double *iv = inv + row * n;
    for (int64_t j = 0; j < n; ++j) acc += iv[j] * (double)g[j * R + r];
    u[idx] = (T)acc;
}

// ---------------------------------------------------------------- layout conversion
// pack: out[i * R + r] = in[r * n + i] (r < nrhs); unpack: out[r * n + i] = in[i * R + r].
// 32 x 32 tiles through shared memory, blockIdx.x over rows i, blockIdx.y over columns r.
__global__ void pack_kernel(int64_t n, int nrhs, int R, const double *__restrict__ in, double *__restrict__ out) {
    __shared__ double tile[32][33];
    const int64_t i0 = (int64_t)blockIdx.x * 32;
    const int r0 = blockIdx.y * 32;
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int r = r0 + dy;
        const int64_t i = i0 + threadIdx.x;
        if (r < nrhs && i < n) tile[dy][threadIdx.x] = in[(int64_t)r * n + i];
    }
    __syncthreads();
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int64_t i = i0 + dy;
        const int r = r0 + threadIdx.x;
        if (r < nrhs && i < n) out[i * R + r] = tile[threadIdx.x][dy];
    }
}

__global__ void unpack_kernel(int64_t n, int nrhs, int R, const double *__restrict__ in, double *__restrict__ out) {
    __shared__ double tile[32][33];
    const int64_t i0 = (int64_t)blockIdx.x * 32;
    const int r0 = blockIdx.y * 32;
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int64_t i = i0 + dy;
        const int r = r0 + threadIdx.x;
        if (r < nrhs && i < n) tile[dy][threadIdx.x] = in[i * R + r];
    }
    __syncthreads();
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int r = r0 + dy;
        const int64_t i = i0 + threadIdx.x;
        if (r < nrhs && i < n) out[(int64_t)r * n + i] = tile[threadIdx.x][dy];
    }
}

template <class Ti, class To>
__global__ void convert_kernel(const Ti *__restrict__ x, To *__restrict__ y, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] = (To)x[i];
}

// ---------------------------------------------------------------- Krylov (FP64)
// Per-column reduction of acc over the threads of a block that share a column
// (thread t holds column t % R), written to partials[(i*R + r)*gridDim.x + block].
__device__ void col_reduce_store(double v, int i, int R, double *partials, double *red) {
    red[threadIdx.x] = v;
    __syncthreads();
    if ((int)threadIdx.x < R) {
        double s = 0.0;
        for (int t = threadIdx.x; t < (int)blockDim.x; t += R) s += red[t];
        partials[((size_t)i * R + threadIdx.x) * gridDim.x + blockIdx.x] = s;
    }
    __syncthreads();
}

// partials of h_{i,r} = <V_i(:, r), w(:, r)> for vectors i0 = 16*blockIdx.y .. (nvb <= NVB)
template <int NVB>
__global__ void __launch_bounds__(MT)
dots_m_kernel(const double *__restrict__ V, int nv, int64_t ld, const double *__restrict__ w, int64_t n, int R,
              double *__restrict__ partials) {
    __shared__ double red[MT];
    const int i0 = 16 * blockIdx.y;
    const int nvb = min(nv - i0, NVB);
    const double *Vb = V + (size_t)i0 * ld;
    double acc[NVB];
#pragma unroll
    for (int i = 0; i < NVB; ++i) acc[i] = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const double we = w[e];
#pragma unroll
        for (int i = 0; i < NVB; ++i)
            if (i < nvb) acc[i] = fma(Vb[(size_t)i * ld + e], we, acc[i]);
    }
#pragma unroll
    for (int i = 0; i < NVB; ++i)
        if (i < nvb) col_reduce_store(acc[i], i0 + i, R, partials, red);   // nvb is uniform over the block
}

// w(:, r) -= Σ_i h_{i,r} V_i(:, r); MODE 1: also partials of <V_i, w_new> per column (nv <= NVB <= 8);
// MODE 2: partials of |w_new(:, r)|^2; MODE 0: update only
template <int NVB, int MODE>
__global__ void __launch_bounds__(MT)
update_dots_m_kernel(const double *__restrict__ V, int nv, int64_t ld, double *__restrict__ w, int64_t n, int R,
                     const double *__restrict__ h, double *__restrict__ partials) {
    __shared__ double hs[MAXVM * 64];
    __shared__ double red[MT];
    for (int i = threadIdx.x; i < nv * R; i += blockDim.x) hs[i] = h[i];
    __syncthreads();
    const int r = threadIdx.x % R;
    constexpr int NA = MODE == 1 ? NVB : 1;
    double acc[NA];
#pragma unroll
    for (int i = 0; i < NA; ++i) acc[i] = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        double we = w[e];
        if (MODE == 1 && NVB <= 16) {
            // basis values stay in registers between the update and the dots
            double vr[NVB];
#pragma unroll
            for (int i = 0; i < NVB; ++i) vr[i] = i < nv ? V[(size_t)i * ld + e] : 0.0;
#pragma unroll
            for (int i = 0; i < NVB; ++i)
                if (i < nv) we = fma(-hs[i * R + r], vr[i], we);
            w[e] = we;
#pragma unroll
            for (int i = 0; i < NVB; ++i)
                if (i < nv) acc[i] = fma(vr[i], we, acc[i]);
        } else if (MODE == 1) {
            // too many for registers: the second read of V_i(e) is served by L1
#pragma unroll
            for (int i = 0; i < NVB; ++i)
                if (i < nv) we = fma(-hs[i * R + r], V[(size_t)i * ld + e], we);
            w[e] = we;
#pragma unroll
            for (int i = 0; i < NVB; ++i)
                if (i < nv) acc[i] = fma(V[(size_t)i * ld + e], we, acc[i]);
        } else {
#pragma unroll 4
            for (int i = 0; i < nv; ++i) we = fma(-hs[i * R + r], V[(size_t)i * ld + e], we);
            w[e] = we;
            if (MODE == 2) acc[0] = fma(we, we, acc[0]);
        }
    }
    if (MODE == 1) {
#pragma unroll
        for (int i = 0; i < NVB; ++i)
            if (i < nv) col_reduce_store(acc[i], i, R, partials, red);   // nv is uniform over the block
    } else if (MODE == 2) {
        col_reduce_store(acc[0], 0, R, partials, red);
    }
}

// small[r*stride + off + i] = Σ_b partials[(i*R + r)*nb + b], and hbuf[i*R + r] the same when given
__global__ void reduce_partials_m_kernel(const double *__restrict__ partials, int nv, int R, int nb,
                                         double *__restrict__ small, int stride, int off, double *__restrict__ hbuf) {
    const int ir = blockIdx.x;
    if (ir >= nv * R) return;
    const int i = ir / R, r = ir % R;
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += 32) s += partials[(size_t)ir * nb + b];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) {
        small[(size_t)r * stride + off + i] = s;
        if (hbuf) hbuf[ir] = s;
    }
}

// Givens step j of every column's least-squares problem (one thread per column)
__global__ void givens_m_kernel(double *small, int stride, int j, int Rst, int R) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    SmallLayout Ly{Rst};
    double *sm = small + (size_t)r * stride;
    double *H = sm + Ly.H(), *cs = sm + Ly.cs(), *sn = sm + Ly.sn(), *g = sm + Ly.g();
    double col[MAXVM + 1];
    for (int i = 0; i <= j; ++i) col[i] = sm[Ly.h1() + i] + sm[Ly.h2() + i];
    const double hn = sqrt(fmax(sm[Ly.nrm2()], 0.0));
    col[j + 1] = hn;
    for (int i = 0; i < j; ++i) {
        const double a = col[i], b = col[i + 1];
        col[i] = cs[i] * a + sn[i] * b;
        col[i + 1] = -sn[i] * a + cs[i] * b;
    }
    const double den = hypot(col[j], col[j + 1]);
    const double c = den > 0.0 ? col[j] / den : 1.0, s = den > 0.0 ? col[j + 1] / den : 0.0;
    cs[j] = c;
    sn[j] = s;
    col[j] = den;
    col[j + 1] = 0.0;
    g[j + 1] = -s * g[j];
    g[j] = c * g[j];
    for (int i = 0; i <= j + 1; ++i) H[(size_t)j * (Rst + 1) + i] = col[i];
    sm[Ly.res()] = fabs(g[j + 1]);
    sm[Ly.hn()] = hn;
}

// v = w / hn_r per column
__global__ void scale_next_m_kernel(const double *__restrict__ w, double *__restrict__ v, int64_t n, int R,
                                    const double *__restrict__ small, int stride, int hn_off) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    const double hn = small[(size_t)(e % R) * stride + hn_off];
    v[e] = hn > 0.0 ? w[e] / hn : 0.0;
}

// v0 = r / beta_r and g_r = beta_r e_1 per column
__global__ void init_cycle_m_kernel(const double *__restrict__ rr, double *__restrict__ v0, int64_t n, int R,
                                    double *__restrict__ small, int stride, int Rst) {
    SmallLayout Ly{Rst};
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < n) {
        const double beta = sqrt(fmax(small[(size_t)(e % R) * stride + Ly.nrm2()], 0.0));
        v0[e] = beta > 0.0 ? rr[e] / beta : 0.0;
    }
    if (e < (int64_t)R * (Rst + 1)) {
        const int r = (int)(e / (Rst + 1)), i = (int)(e % (Rst + 1));
        double *sm = small + (size_t)r * stride;
        sm[Ly.g() + i] = i == 0 ? sqrt(fmax(sm[Ly.nrm2()], 0.0)) : 0.0;
    }
}

// y_r = H_r^{-1} g_r with m_r columns (one thread per column)
__global__ void backsolve_m_kernel(double *small, int stride, const int *__restrict__ m_r, int Rst, int R) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    SmallLayout Ly{Rst};
    double *sm = small + (size_t)r * stride;
    const double *H = sm + Ly.H(), *g = sm + Ly.g();
    double *y = sm + Ly.y();
    const int m = m_r[r];
    for (int i = m - 1; i >= 0; --i) {
        double s = g[i];
        for (int p = i + 1; p < m; ++p) s -= H[(size_t)p * (Rst + 1) + i] * y[p];
        y[i] = s / H[(size_t)i * (Rst + 1) + i];
    }
}

// x(:, r) += Σ_{j < m_r} y_{r,j} Z_j(:, r)
__global__ void update_x_m_kernel(const double *__restrict__ Z, int mmax, int64_t ld,
                                  const double *__restrict__ small, int stride, int y_off,
                                  const int *__restrict__ m_r, double *__restrict__ x, int64_t n, int R) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int r = (int)(e % R);
    const int m = min(m_r[r], mmax);
    const double *y = small + (size_t)r * stride + y_off;
    double s = x[e];
    for (int j = 0; j < m; ++j) s += y[j] * Z[(size_t)j * ld + e];
    x[e] = s;
}

// ---------------------------------------------------------------- Uzawa (FP64)
// g = F + B^* p per column (only the m = 0 normal moment of each facet carries the flux)
__global__ void uzawa_rhs_m_kernel(int64_t n_int, int dpf, int R, const int *__restrict__ facet_adj,
                                   const double *__restrict__ cell_d, const double *__restrict__ F,
                                   const double *__restrict__ p, double *__restrict__ g) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n_int * dpf * R) return;
    const int64_t row = idx / R;
    const int r = (int)(idx - row * R);
    const int64_t i = row / dpf;
    const int d = (int)(row - i * dpf);
    double v = F[idx];
    if (d == 0)
        for (int q = 0; q < 2; ++q) {
            const int adj = facet_adj[2 * i + q];
            if (adj < 0) continue;
            const int64_t c = adj >> 2;
            const int lf = adj & 3;
            v += p[c * R + r] * cell_d[3 * c + lf];
        }
    g[idx] = v;
}

// p_K <- p_K - eps^{-1} (div u)_K per column, with per-column partials of
// Σ|K| dp^2, Σ|K| p^2 and Σ (∫div u)^2
__global__ void __launch_bounds__(MT)
uzawa_update_m_kernel(int64_t nc, int dpf, int R, const int *__restrict__ cell_int,
                      const double *__restrict__ cell_d, const double *__restrict__ area,
                      const double *__restrict__ u, double *__restrict__ p, double gamma, double nu,
                      const double *__restrict__ nu_cell, const int *__restrict__ frozen,
                      double *__restrict__ partials) {
    __shared__ double red[MT];
    double acc[3] = {0.0, 0.0, 0.0};
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nc * R; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / R;
        const int r = (int)(e - c * R);
        if (frozen[r]) continue;
        double du = 0.0;
        for (int f = 0; f < 3; ++f) {
            const int j = cell_int[3 * c + f];
            if (j >= 0) du += cell_d[3 * c + f] * u[((size_t)j * dpf) * R + r];
        }
        const double a = area[c];
        const double dp = gamma * (nu_cell ? nu_cell[c] : nu) * du / a;
        const double pn = p[e] - dp;
        p[e] = pn;
        acc[0] += a * dp * dp;
        acc[1] += a * pn * pn;
        acc[2] += du * du;
    }
    for (int i = 0; i < 3; ++i) col_reduce_store(acc[i], i, R, partials, red);
}

} // namespace

// ================================================================ launchers
// blocks of the grid-stride Krylov kernels (4 per SM); with 256 threads a block
// covers whole rows of every R (a power of two <= 64), so each thread keeps one column
int krylov_m_blocks() { return 608; }

int log2_width(int R) {
    int l = 0;
    while ((1 << l) < R) ++l;
    return l;
}

template <class T>
cudaError_t launch_apply_m(const DevLevel &L, const DevOperator &op, int R, const T *A, const T *x, const T *g, T *y,
                           cudaStream_t s) {
    const int lg = log2_width(R);
    if (L.n_int == 0) return cudaSuccess;
    note_launches(1);
#define HDG_APPLY_M(D, B)                                                                                      \
    case D:                                                                                                    \
        apply_m_kernel<T, D, B><<<nblk((L.n_int * (D / B)) << lg, MT), MT, 0, s>>>(L.n_int, lg, L.facet_adj.p, \
                                                                                L.cell_int.p, A, x, g, y);     \
        break;
    switch (op.dpf) {
        HDG_APPLY_M(2, 2)
        HDG_APPLY_M(4, 4)
        HDG_APPLY_M(6, 2)
        HDG_APPLY_M(8, 4)
        HDG_APPLY_M(10, 2)
    default: return cudaErrorInvalidValue;
    }
#undef HDG_APPLY_M
    return cudaGetLastError();
}

cudaError_t launch_apply_df_m(const DevLevel &L, const DevOperator &op, int R, const float *Ahi, const float *Alo,
                              const double *x, float2 *xsplit, const double *g, double *y, cudaStream_t s) {
    const int lg = log2_width(R);
    if (L.n_int == 0) return cudaSuccess;
    const int64_t nx = (L.n_int * op.dpf) << lg;
    note_launches(2);
    split_x_kernel<<<nblk(nx, MT), MT, 0, s>>>(x, xsplit, nx);
    const float2 *xp = xsplit;
#define HDG_APPLY_DF(D, B)                                                                                     \
    case D:                                                                                                    \
        apply_df_m_kernel<D, B><<<nblk((L.n_int * (D / B)) << lg, MT), MT, 0, s>>>(L.n_int, lg, L.facet_adj.p, \
                                                                                L.cell_int.p, Ahi, Alo, xp, g, y); \
        break;
    switch (op.dpf) {
        HDG_APPLY_DF(2, 2)
        HDG_APPLY_DF(4, 4)
        HDG_APPLY_DF(6, 2)
        HDG_APPLY_DF(8, 4)
        HDG_APPLY_DF(10, 2)
    default: return cudaErrorInvalidValue;
    }
#undef HDG_APPLY_DF
    return cudaGetLastError();
}

cudaError_t launch_split_lo(const double *A, const float *hi, float *lo, int64_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    note_launches(1);
    split_lo_kernel<<<nblk(n, MT), MT, 0, s>>>(A, hi, lo, n);
    return cudaGetLastError();
}

// the closed-form sweep (levels with patch_cext; FP32 with the AL split) reads dpf instead of
// n_loc columns per row and keeps the star cells' outside fluxes after the index tables
static bool gs_m_closed(const DevLevel &L, const DevOperator &op, bool fp32) {
    return L.patch_cext.p && (!fp32 || (op.swQ.p && op.swA00.p));
}

size_t gs_m_smem(const DevLevel &L, const DevOperator &op, int R, size_t word) {
    const size_t nx = gs_m_closed(L, op, word == sizeof(float)) ? (size_t)op.dpf : (size_t)op.nloc;
    return word * (((size_t)L.pc_max * nx + op.np_max) * R + (size_t)L.pf_max * 2 * nx * op.dpf +
                   (size_t)op.np_max * op.np_max + (size_t)L.pc_max * R) +
           sizeof(int) * (((size_t)L.pc_max * 3 + (size_t)L.pf_max * 5 + 3) & ~(size_t)3);
}

namespace {
template <class T, int DPF, int RB>
cudaError_t gs_m_launch(const DevLevel &L, const DevOperator &op, int R, const T *A, const T *Pinv, int colour,
                        const T *g, T *u, int nt, cudaStream_t s) {
    const int p0 = L.colour_ptr[colour], p1 = L.colour_ptr[colour + 1];
    if (p1 <= p0) return cudaSuccess;
    const size_t smem = gs_m_smem(L, op, R, sizeof(T));
    // closed form on levels with the outside-facet table: FP64 directly, FP32 with the AL split
    // (the batched sweeps run on the operator's own copies, Af / Pinvf in FP32)
    const bool fp32 = std::is_same<T, float>::value;
    auto kern = gs_m_closed(L, op, fp32) ? gs_m_kernel<T, DPF, RB, true> : gs_m_kernel<T, DPF, RB, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    note_launches(1);
    kern<<<p1 - p0, nt, smem, s>>>(p0, p1, L.pf_max, L.pc_max, op.np_max, log2_width(R), L.patch_nf.p,
                                   L.patch_facets.p, L.patch_nc.p, L.patch_cells.p, L.patch_slot_src.p, L.cell_int.p,
                                   L.patch_cext.p, fp32 ? op.swQ.p : nullptr, fp32 ? op.swA00.p : nullptr,
                                   L.cell_d.p, A, Pinv, g, u);
    return cudaGetLastError();
}

// rows per thread (RB, a divisor of dpf) of the batched sweep: the tile shape the
// autotuner chooses from; 0 picks the default of each dpf
template <class T, int DPF>
cudaError_t gs_m_rb(const DevLevel &L, const DevOperator &op, int R, const T *A, const T *Pinv, int colour,
                    const T *g, T *u, int rb, int nt, cudaStream_t s) {
    if (rb == 0) rb = (DPF % 4 == 0) ? 4 : 2;
    if (DPF % rb != 0) return cudaErrorInvalidValue;
    switch (rb) {
    case 1: return gs_m_launch<T, DPF, 1>(L, op, R, A, Pinv, colour, g, u, nt, s);
    case 2: return gs_m_launch<T, DPF, (DPF % 2 == 0 ? 2 : 1)>(L, op, R, A, Pinv, colour, g, u, nt, s);
    case 4: return gs_m_launch<T, DPF, (DPF % 4 == 0 ? 4 : 1)>(L, op, R, A, Pinv, colour, g, u, nt, s);
    default: return cudaErrorInvalidValue;
    }
}
} // namespace

template <class T>
cudaError_t launch_gs_colour_m(const DevLevel &L, const DevOperator &op, int R, const T *A, const T *Pinv,
                               int colour, const T *g, T *u, cudaStream_t s, int rb, int nt) {
    if (nt == 0) nt = MT;
    if (nt % 32 != 0 || nt < 32 || nt > MT) return cudaErrorInvalidValue;   // MT: the launch bound
    switch (op.dpf) {
    case 2: return gs_m_rb<T, 2>(L, op, R, A, Pinv, colour, g, u, rb, nt, s);
    case 4: return gs_m_rb<T, 4>(L, op, R, A, Pinv, colour, g, u, rb, nt, s);
    case 6: return gs_m_rb<T, 6>(L, op, R, A, Pinv, colour, g, u, rb, nt, s);
    case 8: return gs_m_rb<T, 8>(L, op, R, A, Pinv, colour, g, u, rb, nt, s);
    case 10: return gs_m_rb<T, 10>(L, op, R, A, Pinv, colour, g, u, rb, nt, s);
    default: return cudaErrorInvalidValue;
    }
}

template <class T>
cudaError_t launch_hp_restrict_m(int k, int64_t n_int, int R, const T *r, T *r0, cudaStream_t s) {
    if (n_int == 0) return cudaSuccess;
    note_launches(1);
    hp_restrict_m_kernel<T><<<nblk(n_int * R, MT), MT, 0, s>>>(k, n_int, R, r, r0);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_hp_prolong_add_m(int k, int64_t n_int, int R, const T *d0, T *u, cudaStream_t s) {
    if (n_int == 0) return cudaSuccess;
    note_launches(1);
    hp_prolong_m_kernel<T><<<nblk(n_int * R, MT), MT, 0, s>>>(k, n_int, R, d0, u);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_prolong_add_m(const DevLevel &F, const DevLevel &C, int R, const T *W, const T *Hm, const T *uc,
                                 T *tmp, T *uf, cudaStream_t s) {
    if (F.nB > 0) {
        note_launches(1);
        prolong_B_m_kernel<T><<<nblk(F.nB * R, MT), MT, 0, s>>>(F.nB, R, F.tr_fineB.p, F.tr_fineB_src.p,
                                                               C.cell_int.p, W, uc, tmp, uf);
    }
    if (F.nc_coarse > 0) {
        note_launches(1);
        prolong_T_m_kernel<T><<<nblk(F.nc_coarse * R, MT), MT, 0, s>>>(F.nc_coarse, R, F.tr_slots.p, Hm, tmp, uf);
    }
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_restrict_m(const DevLevel &F, const DevLevel &C, int R, const T *W, const T *Hm, const T *rf,
                              T *t1, T *t2, T *rc, cudaStream_t s) {
    if (F.nc_coarse > 0) {
        note_launches(2);
        restrict_T_m_kernel<T><<<nblk(F.nc_coarse * R, MT), MT, 0, s>>>(F.nc_coarse, R, F.tr_slots.p, Hm, rf, t1);
        restrict_B_m_kernel<T><<<nblk(F.nc_coarse * R, MT), MT, 0, s>>>(F.nc_coarse, R, F.tr_slots.p, F.tr_nbr.p,
                                                                        W, rf, t1, t2);
    }
    if (C.n_int > 0) {
        note_launches(1);
        restrict_C_m_kernel<T><<<nblk(C.n_int * R, MT), MT, 0, s>>>(C.n_int, R, C.facet_adj.p, t2, rc);
    }
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_coarse_apply_m(const double *inv, int64_t n, int R, const T *g, T *u, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    note_launches(1);
    coarse_m_kernel<T><<<nblk(n * R, MT), MT, 0, s>>>(inv, n, R, g, u);
    return cudaGetLastError();
}

cudaError_t launch_pack_m(const double *in, int nrhs, int64_t n, int R, double *out, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    if (R > nrhs) {
        cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * (size_t)n * R, s);
        if (e != cudaSuccess) return e;
    }
    note_launches(1);
    pack_kernel<<<dim3(nblk(n, 32), nblk(nrhs, 32)), dim3(32, 8), 0, s>>>(n, nrhs, R, in, out);
    return cudaGetLastError();
}

cudaError_t launch_unpack_m(const double *in, int nrhs, int64_t n, int R, double *out, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    note_launches(1);
    unpack_kernel<<<dim3(nblk(n, 32), nblk(nrhs, 32)), dim3(32, 8), 0, s>>>(n, nrhs, R, in, out);
    return cudaGetLastError();
}

template <class Ti, class To>
cudaError_t launch_convert_m(const Ti *x, To *y, int64_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    note_launches(1);
    convert_kernel<Ti, To><<<nblk(n, MT), MT, 0, s>>>(x, y, n);
    return cudaGetLastError();
}

cudaError_t launch_dots_m(const double *V, int nv, int64_t ld, const double *w, int64_t n, int R, double *partials,
                          cudaStream_t s) {
    if (nv <= 0) return cudaSuccess;
    const int nb = krylov_m_blocks();
    note_launches(1);
    dim3 grid(nb, (nv + 15) / 16);
    if (nv <= 1) dots_m_kernel<1><<<grid, MT, 0, s>>>(V, nv, ld, w, n, R, partials);
    else if (nv <= 4) dots_m_kernel<4><<<grid, MT, 0, s>>>(V, nv, ld, w, n, R, partials);
    else if (nv <= 8) dots_m_kernel<8><<<grid, MT, 0, s>>>(V, nv, ld, w, n, R, partials);
    else dots_m_kernel<16><<<grid, MT, 0, s>>>(V, nv, ld, w, n, R, partials);
    return cudaGetLastError();
}

cudaError_t launch_update_dots_m(const double *V, int nv, int64_t ld, double *w, int64_t n, int R, const double *h,
                                 double *partials, int mode, cudaStream_t s) {
    const int nb = krylov_m_blocks();
    note_launches(1);
    if (mode == 1) {
        if (nv <= 1) update_dots_m_kernel<1, 1><<<nb, MT, 0, s>>>(V, nv, ld, w, n, R, h, partials);
        else if (nv <= 4) update_dots_m_kernel<4, 1><<<nb, MT, 0, s>>>(V, nv, ld, w, n, R, h, partials);
        else if (nv <= 8) update_dots_m_kernel<8, 1><<<nb, MT, 0, s>>>(V, nv, ld, w, n, R, h, partials);
        else if (nv <= 16) update_dots_m_kernel<16, 1><<<nb, MT, 0, s>>>(V, nv, ld, w, n, R, h, partials);
        else if (nv <= 32) update_dots_m_kernel<32, 1><<<nb, MT, 0, s>>>(V, nv, ld, w, n, R, h, partials);
        else {
            // update only, then the dots of the new w in chunks of 16
            update_dots_m_kernel<1, 0><<<nb, MT, 0, s>>>(V, nv, ld, w, n, R, h, partials);
            return launch_dots_m(V, nv, ld, w, n, R, partials, s);
        }
    } else if (mode == 2) {
        update_dots_m_kernel<1, 2><<<nb, MT, 0, s>>>(V, nv, ld, w, n, R, h, partials);
    } else {
        update_dots_m_kernel<1, 0><<<nb, MT, 0, s>>>(V, nv, ld, w, n, R, h, partials);
    }
    return cudaGetLastError();
}

cudaError_t launch_reduce_partials_m(const double *partials, int nv, int R, double *small, int stride, int off,
                                     double *hbuf, cudaStream_t s) {
    note_launches(1);
    reduce_partials_m_kernel<<<nv * R, 32, 0, s>>>(partials, nv, R, krylov_m_blocks(), small, stride, off, hbuf);
    return cudaGetLastError();
}

cudaError_t launch_givens_m(double *small, int stride, int j, int Rst, int R, cudaStream_t s) {
    note_launches(1);
    givens_m_kernel<<<1, 64, 0, s>>>(small, stride, j, Rst, R);
    return cudaGetLastError();
}

cudaError_t launch_scale_next_m(const double *w, double *v, int64_t n, int R, const double *small, int stride,
                                int hn_off, cudaStream_t s) {
    note_launches(1);
    scale_next_m_kernel<<<nblk(n, MT), MT, 0, s>>>(w, v, n, R, small, stride, hn_off);
    return cudaGetLastError();
}

cudaError_t launch_init_cycle_m(const double *r, double *v0, int64_t n, int R, double *small, int stride, int Rst,
                                cudaStream_t s) {
    const int64_t m = std::max<int64_t>(n, (int64_t)R * (Rst + 1));
    note_launches(1);
    init_cycle_m_kernel<<<nblk(m, MT), MT, 0, s>>>(r, v0, n, R, small, stride, Rst);
    return cudaGetLastError();
}

cudaError_t launch_solve_update_m(double *small, int stride, const int *m_r, int mmax, int Rst, const double *Z,
                                  int64_t ld, double *x, int64_t n, int R, cudaStream_t s) {
    if (mmax <= 0) return cudaSuccess;
    SmallLayout Ly{Rst};
    note_launches(2);
    backsolve_m_kernel<<<1, 64, 0, s>>>(small, stride, m_r, Rst, R);
    update_x_m_kernel<<<nblk(n, MT), MT, 0, s>>>(Z, mmax, ld, small, stride, Ly.y(), m_r, x, n, R);
    return cudaGetLastError();
}

cudaError_t launch_uzawa_rhs_m(const DevLevel &L, int k, int R, const double *F, const double *p, double *g,
                               cudaStream_t s) {
    const int dpf = 2 * (k + 1);
    const int64_t n = L.n_int * dpf * R;
    if (n == 0) return cudaSuccess;
    note_launches(1);
    uzawa_rhs_m_kernel<<<nblk(n, MT), MT, 0, s>>>(L.n_int, dpf, R, L.facet_adj.p, L.cell_d.p, F, p, g);
    return cudaGetLastError();
}

cudaError_t launch_uzawa_update_m(const DevLevel &L, int k, int R, const double *u, double *p, double gamma, double nu,
                                  const double *nu_cell, const int *frozen, double *partials, cudaStream_t s) {
    note_launches(1);
    uzawa_update_m_kernel<<<krylov_m_blocks(), MT, 0, s>>>(L.nc, 2 * (k + 1), R, L.cell_int.p, L.cell_d.p,
                                                            L.cell_area.p, u, p, gamma, nu, nu_cell, frozen,
                                                            partials);
    return cudaGetLastError();
}

#define HDG_MULTI_INST(T)                                                                                          \
    template cudaError_t launch_apply_m<T>(const DevLevel &, const DevOperator &, int, const T *, const T *,        \
                                           const T *, T *, cudaStream_t);                                          \
    template cudaError_t launch_gs_colour_m<T>(const DevLevel &, const DevOperator &, int, const T *, const T *,    \
                                               int, const T *, T *, cudaStream_t, int, int);                       \
    template cudaError_t launch_hp_restrict_m<T>(int, int64_t, int, const T *, T *, cudaStream_t);                  \
    template cudaError_t launch_hp_prolong_add_m<T>(int, int64_t, int, const T *, T *, cudaStream_t);               \
    template cudaError_t launch_prolong_add_m<T>(const DevLevel &, const DevLevel &, int, const T *, const T *,     \
                                                 const T *, T *, T *, cudaStream_t);                               \
    template cudaError_t launch_restrict_m<T>(const DevLevel &, const DevLevel &, int, const T *, const T *,        \
                                              const T *, T *, T *, T *, cudaStream_t);                             \
    template cudaError_t launch_coarse_apply_m<T>(const double *, int64_t, int, const T *, T *, cudaStream_t);
HDG_MULTI_INST(double)
HDG_MULTI_INST(float)
#undef HDG_MULTI_INST
template cudaError_t launch_convert_m<double, float>(const double *, float *, int64_t, cudaStream_t);
template cudaError_t launch_convert_m<float, double>(const float *, double *, int64_t, cudaStream_t);

} // namespace hdg
