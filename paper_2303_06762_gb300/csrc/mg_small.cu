// Algorithm 1 (MG_h) on the smallest lowest-order levels in one thread block.
//
// On the coarse levels of a deep hierarchy each colour phase of the block
// Gauss-Seidel smoother touches a few hundred patches, and the variable
// V-cycle doubles the smoothing steps per level (m(l-1) = 2 m(l)), so these
// levels produce most of the launches of a preconditioner application while
// moving little data.  Here one 1024-thread block runs the whole recursion
// below a level Ls (pre-smoothing colour by colour, residual, restriction,
// recursion, the FP64 dense coarse solve, prolongation with harmonic extension,
// post-smoothing in reverse colour order) with a block barrier between steps
// instead of a kernel boundary.  The arithmetic of every step is the one of the
// multi-block kernels in ops.cu (same formulas, same order per unknown).
#include <cuda_runtime.h>

#include "hdg_internal.h"

namespace hdg {
namespace {

template <class T>
__device__ void blk_fill(T *u, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) u[i] = T(0);
}

template <class T>
__device__ void blk_gs_colour(const SmallLevel<T> &L, int c, const T *g, T *u, T *rs) {
    const int p0 = L.colour_ptr[c], p1 = L.colour_ptr[c + 1];
    const int items = (p1 - p0) * L.np_max;
    for (int w = threadIdx.x; w < items; w += blockDim.x) {
        const int p = p0 + w / L.np_max, t = w % L.np_max;
        const int np = 2 * L.patch_nf[p];
        if (t >= np) continue;
        const int js = t >> 1, d = t & 1;
        const int F = L.patch_facets[p * L.pf_max + js];
        T acc = g[2 * F + d];
        for (int q = 0; q < 2; ++q) {
            const int src = L.slot_src[(p * L.pf_max + js) * 2 + q];
            const int si = src >> 2, lf = src & 3;
            const int cell = L.patch_cells[p * L.pc_max + si];
            const T *Ac = L.A + (size_t)cell * 36 + 2 * lf + d;
#pragma unroll
            for (int col = 0; col < 6; ++col) {
                const int j = L.cell_int[3 * cell + col / 2];
                if (j >= 0) acc -= Ac[col * 6] * u[2 * j + (col & 1)];
            }
        }
        rs[w] = acc;
    }
    __syncthreads();
    for (int w = threadIdx.x; w < items; w += blockDim.x) {
        const int p = p0 + w / L.np_max, t = w % L.np_max;
        const int np = 2 * L.patch_nf[p];
        if (t >= np) continue;
        const T *Pi = L.Pinv + (size_t)p * L.np_max * L.np_max;
        const T *rp = rs + (w / L.np_max) * L.np_max;
        T acc = 0;
        for (int j = 0; j < np; ++j) acc += Pi[j * L.np_max + t] * rp[j];
        const int F = L.patch_facets[p * L.pf_max + (t >> 1)];
        u[2 * F + (t & 1)] += acc;
    }
    __syncthreads();
}

template <class T>
__device__ void blk_sweep(const SmallLevel<T> &L, const T *g, T *u, bool reverse, T *rs) {
    for (int i = 0; i < L.n_colours; ++i) blk_gs_colour(L, reverse ? L.n_colours - 1 - i : i, g, u, rs);
}

template <class T>
__device__ void blk_residual(const SmallLevel<T> &L, const T *g, const T *u, T *r) {
    for (int idx = threadIdx.x; idx < 2 * L.n_int; idx += blockDim.x) {
        const int i = idx >> 1, d = idx & 1;
        T acc = 0;
        for (int q = 0; q < 2; ++q) {
            const int adj = L.facet_adj[2 * i + q];
            if (adj < 0) continue;
            const int cell = adj >> 2, lf = adj & 3;
            const T *Ac = L.A + (size_t)cell * 36 + 2 * lf + d;
#pragma unroll
            for (int col = 0; col < 6; ++col) {
                const int j = L.cell_int[3 * cell + col / 2];
                if (j >= 0) acc += Ac[col * 6] * u[2 * j + (col & 1)];
            }
        }
        r[idx] = g[idx] - acc;
    }
    __syncthreads();
}

// g_c = (I_{l-1}^l)^T r_f  (F = fine level l, C = coarse level l-1)
template <class T>
__device__ void blk_restrict(const SmallLevel<T> &F, const SmallLevel<T> &C, const T *rf, T *gc) {
    for (int P = threadIdx.x; P < F.ncc; P += blockDim.x) {
        T rT[6];
        for (int t = 0; t < 6; ++t) rT[t] = rf[2 * F.tr_slots[9 * P + 6 + t / 2] + (t & 1)];
        const T *Hk = F.H + (size_t)P * 72;
        for (int c = 0; c < 12; ++c) {
            T acc = 0;
            for (int t = 0; t < 6; ++t) acc += Hk[t * 12 + c] * rT[t];
            F.ct1[12 * P + c] = acc;
        }
    }
    __syncthreads();
    for (int P = threadIdx.x; P < F.ncc; P += blockDim.x) {
        T z[12];
        for (int s = 0; s < 6; ++s) {
            const int i = F.tr_slots[9 * P + s];
            if (i < 0) { z[2 * s] = z[2 * s + 1] = 0; continue; }
            const int nb = F.tr_nbr[6 * P + s];
            const int Q = nb >> 4, s2 = nb & 15;
            for (int c = 0; c < 2; ++c)
                z[2 * s + c] = rf[2 * i + c] + F.ct1[12 * P + 2 * s + c] + F.ct1[12 * Q + 2 * s2 + c];
        }
        const T *Wk = F.W + (size_t)P * 72;
        for (int col = 0; col < 6; ++col) {
            T acc = 0;
            for (int row = 0; row < 12; ++row) acc += Wk[row * 6 + col] * z[row];
            F.ct2[6 * P + col] = acc;
        }
    }
    __syncthreads();
    for (int G = threadIdx.x; G < C.n_int; G += blockDim.x) {
        T a0 = 0, a1 = 0;
        for (int q = 0; q < 2; ++q) {
            const int adj = C.facet_adj[2 * G + q];
            const int K = adj >> 2, lf = adj & 3;
            a0 += F.ct2[6 * K + 2 * lf];
            a1 += F.ct2[6 * K + 2 * lf + 1];
        }
        gc[2 * G] = a0;
        gc[2 * G + 1] = a1;
    }
    __syncthreads();
}

// u_f += I_{l-1}^l u_c
template <class T>
__device__ void blk_prolong_add(const SmallLevel<T> &F, const SmallLevel<T> &C, const T *uc, T *uf, T *tmp) {
    for (int b = threadIdx.x; b < F.nB; b += blockDim.x) {
        T v0 = 0, v1 = 0;
        for (int q = 0; q < 2; ++q) {
            const int src = F.tr_fineB_src[2 * b + q];
            const int P = src >> 4, s = src & 15;
            const T *Wk = F.W + (size_t)P * 72;
            for (int fp = 0; fp < 3; ++fp) {
                const int j = C.cell_int[3 * P + fp];
                if (j < 0) continue;
                for (int cq = 0; cq < 2; ++cq) {
                    const T u = uc[2 * j + cq];
                    v0 += Wk[(2 * s) * 6 + 2 * fp + cq] * u;
                    v1 += Wk[(2 * s + 1) * 6 + 2 * fp + cq] * u;
                }
            }
        }
        const int i = F.tr_fineB[b];
        tmp[2 * i] = v0;
        tmp[2 * i + 1] = v1;
        uf[2 * i] += v0;
        uf[2 * i + 1] += v1;
    }
    __syncthreads();
    for (int P = threadIdx.x; P < F.ncc; P += blockDim.x) {
        T bb[12];
        for (int s = 0; s < 6; ++s) {
            const int i = F.tr_slots[9 * P + s];
            bb[2 * s] = i >= 0 ? tmp[2 * i] : T(0);
            bb[2 * s + 1] = i >= 0 ? tmp[2 * i + 1] : T(0);
        }
        const T *Hk = F.H + (size_t)P * 72;
        for (int t = 0; t < 6; ++t) {
            T acc = 0;
            for (int c = 0; c < 12; ++c) acc += Hk[t * 12 + c] * bb[c];
            uf[2 * F.tr_slots[9 * P + 6 + t / 2] + (t & 1)] += acc;
        }
    }
    __syncthreads();
}

// u_0 = inv g_0 in FP64 (one warp per row)
template <class T>
__device__ void blk_coarse(const SmallParams<T> &S) {
    const SmallLevel<T> &L0 = S.lv[0];
    const int n = 2 * L0.n_int;
    for (int i = threadIdx.x; i < n; i += blockDim.x) S.g0d[i] = (double)L0.g[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int row = wid; row < n; row += nw) {
        double acc = 0.0;
        for (int j = lane; j < n; j += 32) acc += S.inv[(size_t)row * n + j] * S.g0d[j];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) L0.u[row] = (T)acc;
    }
    __syncthreads();
}

// MG_h(l_top, g, u, m, q) without recursion: an explicit walk down and up the
// levels, where visit[l] counts the coarse-grid corrections done at level l (q of
// them: 1 for the V-cycle, 2 for the W-cycle).  Every thread holds the same state.
template <class T>
__device__ void blk_mg(const SmallParams<T> &S, int top, int m_top, bool zero_top, T *rs) {
    int mlev[SMALL_MAX_LEVELS];
    int visit[SMALL_MAX_LEVELS];
    int l = top;
    mlev[top] = m_top;
    bool zero = zero_top;
    bool descending = true;
    while (true) {
        if (descending) {
            if (l == 0) {
                blk_coarse(S);
                descending = false;
                l = 1;
                continue;
            }
            const SmallLevel<T> &L = S.lv[l];
            const SmallLevel<T> &C = S.lv[l - 1];
            if (zero) {
                blk_fill(L.u, 2 * L.n_int);
                __syncthreads();
            }
            for (int j = 0; j < mlev[l]; ++j) blk_sweep(L, L.g, L.u, false, rs);
            blk_residual(L, L.g, L.u, L.r);
            blk_restrict(L, C, L.r, C.g);
            visit[l] = 0;
            mlev[l - 1] = S.q == 1 ? mlev[l] * S.growth : mlev[l];
            zero = true;
            l = l - 1;
        } else {
            // returning to level l after one coarse-grid correction from level l-1
            visit[l] += 1;
            if (visit[l] < S.q) {
                zero = false;            // next correction starts from the previous one
                descending = true;
                l = l - 1;
                continue;
            }
            const SmallLevel<T> &L = S.lv[l];
            const SmallLevel<T> &C = S.lv[l - 1];
            blk_prolong_add(L, C, C.u, L.u, L.t);
            for (int j = 0; j < mlev[l]; ++j) blk_sweep(L, L.g, L.u, true, rs);
            if (l == top) break;
            l = l + 1;
        }
    }
}

template <class T>
__global__ void __launch_bounds__(1024) mg_small_kernel(SmallParams<T> S, int l, int m, int zero_init) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T *rs = reinterpret_cast<T *>(smraw);
    blk_mg(S, l, m, zero_init != 0, rs);
}

} // namespace

template <class T>
cudaError_t launch_mg_small(const SmallParams<T> &S, int l, int m, bool zero_init, size_t smem_bytes,
                            cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(mg_small_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_bytes);
    if (e != cudaSuccess) return e;
    note_launches(1);
    mg_small_kernel<T><<<1, 1024, smem_bytes, s>>>(S, l, m, zero_init ? 1 : 0);
    return cudaGetLastError();
}

template cudaError_t launch_mg_small<double>(const SmallParams<double> &, int, int, bool, size_t, cudaStream_t);
template cudaError_t launch_mg_small<float>(const SmallParams<float> &, int, int, bool, size_t, cudaStream_t);

} // namespace hdg
