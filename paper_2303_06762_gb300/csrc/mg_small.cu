// Algorithm 1 (MG_h) on the smallest lowest-order levels in one launch of a
// thread-block cluster.
//
// On the coarse levels of a deep hierarchy each colour phase of the block
// Gauss-Seidel smoother touches a few hundred to a few thousand patches, and
// the variable V-cycle doubles the smoothing steps per level (m(l-1) = 2 m(l)),
// so these levels produce most of the launches of a preconditioner
// application while moving little data.  Here one cluster of up to 16 CTAs
// (one per SM, 1024 threads each) runs the whole recursion below a level Ls:
// pre-smoothing colour by colour, residual, restriction, recursion, the FP64
// dense coarse solve, prolongation with harmonic extension, post-smoothing in
// reverse colour order.  Steps are separated by the hardware cluster barrier
// (barrier.cluster arrive.release / wait.acquire) instead of kernel
// boundaries.  Values written inside the kernel are read through L2 (ld.cg),
// since the CTAs of a cluster sit on different SMs.  Every CTA executes the same
// sequence of barriers: the control flow depends on kernel arguments only.
// The arithmetic of every step is the one of the multi-block kernels in ops.cu
// (same formulas, same order per unknown).
#include <cuda_runtime.h>

#include <algorithm>

#include "hdg_internal.h"

namespace hdg {
namespace {

// the CTAs of the launch acting as one team: a cluster (CL), or one block
template <bool CL>
struct Team {
    int rank, size;
    __device__ int tid() const { return rank * (int)blockDim.x + (int)threadIdx.x; }
    __device__ int nthreads() const { return size * (int)blockDim.x; }
    __device__ void sync() const {
        if constexpr (CL) {
            // non-.aligned forms: no assumption on warp convergence at the call
            asm volatile("barrier.cluster.arrive.release;\n"
                         "barrier.cluster.wait.acquire;\n" ::: "memory");
        } else {
            __syncthreads();
        }
    }
    // values written during the kernel: through L2 when another SM of the cluster may
    // have written them; in a single block its own stores are visible after the barrier
    template <class T>
    __device__ T ld(const T *p) const {
        if constexpr (CL) return __ldcg(p);
        else return *p;
    }
};

template <bool CL>
__device__ __forceinline__ Team<CL> make_team() {
    if constexpr (CL) {
        unsigned r, n;
        asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
        asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(n));
        return Team<CL>{(int)r, (int)n};
    } else {
        return Team<CL>{0, 1};
    }
}

template <class T, bool CL>
__device__ void blk_fill(const Team<CL> &tm, T *u, int n) {
    for (int i = tm.tid(); i < n; i += tm.nthreads()) u[i] = T(0);
}

// one colour phase: CTA `rank` owns the patches p0 + rank + i*size, and its
// residual rows stay in its shared memory between the two passes
template <class T, bool CL>
__device__ void blk_gs_colour(const Team<CL> &tm, const SmallLevel<T> &L, int c, const T *g, T *u, T *rs) {
    const int p0 = L.colour_ptr[c], p1 = L.colour_ptr[c + 1];
    const int mine = (p1 - p0 - tm.rank + tm.size - 1) / tm.size;
    const int items = (mine > 0 ? mine : 0) * L.np_max;
    for (int w = threadIdx.x; w < items; w += blockDim.x) {
        const int p = p0 + tm.rank + (w / L.np_max) * tm.size, t = w % L.np_max;
        const int np = 2 * L.patch_nf[p];
        if (t >= np) continue;
        const int js = t >> 1, d = t & 1;
        const int F = L.patch_facets[p * L.pf_max + js];
        T acc = tm.ld(g + 2 * F + d);
        for (int q = 0; q < 2; ++q) {
            const int src = L.slot_src[(p * L.pf_max + js) * 2 + q];
            const int si = src >> 2, lf = src & 3;
            const int cell = L.patch_cells[p * L.pc_max + si];
            const T *Ac = L.A + (size_t)cell * 36 + lf * 12 + d;
#pragma unroll
            for (int col = 0; col < 6; ++col) {
                const int j = L.cell_int[3 * cell + col / 2];
                if (j >= 0) acc -= Ac[col * 2] * tm.ld(u + 2 * j + (col & 1));
            }
        }
        rs[w] = acc;
    }
    __syncthreads();
    for (int w = threadIdx.x; w < items; w += blockDim.x) {
        const int p = p0 + tm.rank + (w / L.np_max) * tm.size, t = w % L.np_max;
        const int np = 2 * L.patch_nf[p];
        if (t >= np) continue;
        const T *Pi = L.Pinv + (size_t)p * L.np_max * L.np_max;
        const T *rp = rs + (w / L.np_max) * L.np_max;
        T acc = 0;
        for (int j = 0; j < np; ++j) acc += Pi[j * L.np_max + t] * rp[j];
        T *dst = u + 2 * L.patch_facets[p * L.pf_max + (t >> 1)] + (t & 1);
        *dst = tm.ld(dst) + acc;
    }
    tm.sync();
}

template <class T, bool CL>
__device__ void blk_sweep(const Team<CL> &tm, const SmallLevel<T> &L, const T *g, T *u, bool reverse, T *rs) {
    for (int i = 0; i < L.n_colours; ++i) blk_gs_colour(tm, L, reverse ? L.n_colours - 1 - i : i, g, u, rs);
}

template <class T, bool CL>
__device__ void blk_residual(const Team<CL> &tm, const SmallLevel<T> &L, const T *g, const T *u, T *r) {
    for (int idx = tm.tid(); idx < 2 * L.n_int; idx += tm.nthreads()) {
        const int i = idx >> 1, d = idx & 1;
        T acc = 0;
        for (int q = 0; q < 2; ++q) {
            const int adj = L.facet_adj[2 * i + q];
            if (adj < 0) continue;
            const int cell = adj >> 2, lf = adj & 3;
            const T *Ac = L.A + (size_t)cell * 36 + lf * 12 + d;
#pragma unroll
            for (int col = 0; col < 6; ++col) {
                const int j = L.cell_int[3 * cell + col / 2];
                if (j >= 0) acc += Ac[col * 2] * tm.ld(u + 2 * j + (col & 1));
            }
        }
        r[idx] = tm.ld(g + idx) - acc;
    }
    tm.sync();
}

// g_c = (I_{l-1}^l)^T r_f  (F = fine level l, C = coarse level l-1; ct1, ct2 per coarse cell)
template <class T, bool CL>
__device__ void blk_restrict(const Team<CL> &tm, const SmallLevel<T> &F, const SmallLevel<T> &C, const T *rf, T *gc,
                             T *ct1, T *ct2) {
    for (int P = tm.tid(); P < F.ncc; P += tm.nthreads()) {
        T rT[6];
        for (int t = 0; t < 6; ++t) rT[t] = tm.ld(rf + 2 * F.tr_slots[9 * P + 6 + t / 2] + (t & 1));
        const T *Hk = F.H + (size_t)P * 72;
        for (int c = 0; c < 12; ++c) {
            T acc = 0;
            for (int t = 0; t < 6; ++t) acc += Hk[t * 12 + c] * rT[t];
            ct1[12 * P + c] = acc;
        }
    }
    tm.sync();
    for (int P = tm.tid(); P < F.ncc; P += tm.nthreads()) {
        T z[12];
        for (int s = 0; s < 6; ++s) {
            const int i = F.tr_slots[9 * P + s];
            if (i < 0) { z[2 * s] = z[2 * s + 1] = 0; continue; }
            const int nb = F.tr_nbr[6 * P + s];
            const int Q = nb >> 4, s2 = nb & 15;
            for (int c = 0; c < 2; ++c)
                z[2 * s + c] = tm.ld(rf + 2 * i + c) + tm.ld(ct1 + 12 * P + 2 * s + c) + tm.ld(ct1 + 12 * Q + 2 * s2 + c);
        }
        const T *Wk = F.W + (size_t)P * 72;
        for (int col = 0; col < 6; ++col) {
            T acc = 0;
            for (int row = 0; row < 12; ++row) acc += Wk[row * 6 + col] * z[row];
            ct2[6 * P + col] = acc;
        }
    }
    tm.sync();
    for (int G = tm.tid(); G < C.n_int; G += tm.nthreads()) {
        T a0 = 0, a1 = 0;
        for (int q = 0; q < 2; ++q) {
            const int adj = C.facet_adj[2 * G + q];
            const int K = adj >> 2, lf = adj & 3;
            a0 += tm.ld(ct2 + 6 * K + 2 * lf);
            a1 += tm.ld(ct2 + 6 * K + 2 * lf + 1);
        }
        gc[2 * G] = a0;
        gc[2 * G + 1] = a1;
    }
    tm.sync();
}

// u_f += I_{l-1}^l u_c
template <class T, bool CL>
__device__ void blk_prolong_add(const Team<CL> &tm, const SmallLevel<T> &F, const SmallLevel<T> &C, const T *uc, T *uf,
                                T *tmp) {
    for (int b = tm.tid(); b < F.nB; b += tm.nthreads()) {
        T v0 = 0, v1 = 0;
        for (int q = 0; q < 2; ++q) {
            const int src = F.tr_fineB_src[2 * b + q];
            const int P = src >> 4, s = src & 15;
            const T *Wk = F.W + (size_t)P * 72;
            for (int fp = 0; fp < 3; ++fp) {
                const int j = C.cell_int[3 * P + fp];
                if (j < 0) continue;
                for (int cq = 0; cq < 2; ++cq) {
                    const T u = tm.ld(uc + 2 * j + cq);
                    v0 += Wk[(2 * s) * 6 + 2 * fp + cq] * u;
                    v1 += Wk[(2 * s + 1) * 6 + 2 * fp + cq] * u;
                }
            }
        }
        const int i = F.tr_fineB[b];
        tmp[2 * i] = v0;
        tmp[2 * i + 1] = v1;
        uf[2 * i] = tm.ld(uf + 2 * i) + v0;
        uf[2 * i + 1] = tm.ld(uf + 2 * i + 1) + v1;
    }
    tm.sync();
    for (int P = tm.tid(); P < F.ncc; P += tm.nthreads()) {
        T bb[12];
        for (int s = 0; s < 6; ++s) {
            const int i = F.tr_slots[9 * P + s];
            bb[2 * s] = i >= 0 ? tm.ld(tmp + 2 * i) : T(0);
            bb[2 * s + 1] = i >= 0 ? tm.ld(tmp + 2 * i + 1) : T(0);
        }
        const T *Hk = F.H + (size_t)P * 72;
        for (int t = 0; t < 6; ++t) {
            T acc = 0;
            for (int c = 0; c < 12; ++c) acc += Hk[t * 12 + c] * bb[c];
            T *dst = uf + 2 * F.tr_slots[9 * P + 6 + t / 2] + (t & 1);
            *dst = tm.ld(dst) + acc;
        }
    }
    tm.sync();
}

// u_0 = inv g_0 in FP64 (one warp per row)
template <class T, bool CL>
__device__ void blk_coarse(const Team<CL> &tm, const SmallParams<T> &S, const T *g0, T *u0, double *g0d) {
    const int n = 2 * S.lv[0].n_int;
    for (int i = tm.tid(); i < n; i += tm.nthreads()) g0d[i] = (double)tm.ld(g0 + i);
    tm.sync();
    const int lane = threadIdx.x & 31, wid = tm.tid() >> 5, nw = tm.nthreads() >> 5;
    for (int row = wid; row < n; row += nw) {
        double acc = 0.0;
        for (int j = lane; j < n; j += 32) acc += S.inv[(size_t)row * n + j] * tm.ld(g0d + j);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) u0[row] = (T)acc;
    }
    tm.sync();
}

// where the kernel keeps the vectors of one level (global memory, or shared memory)
template <class T>
struct LevelVecs {
    T *g, *u, *r, *t, *c1, *c2;
};

// MG_h(l_top, g, u, m, q) without recursion: an explicit walk down and up the
// levels, where visit[l] counts the coarse-grid corrections done at level l (q of
// them: 1 for the V-cycle, 2 for the W-cycle).  Every thread holds the same state.
template <class T, bool CL>
__device__ void blk_mg(const Team<CL> &tm, const SmallParams<T> &S, const LevelVecs<T> *vv, double *g0d, int top,
                       int m_top, bool zero_top, T *rs) {
    int mlev[SMALL_MAX_LEVELS];
    int visit[SMALL_MAX_LEVELS];
    int l = top;
    mlev[top] = m_top;
    bool zero = zero_top;
    bool descending = true;
    while (true) {
        if (descending) {
            if (l == 0) {
                blk_coarse(tm, S, vv[0].g, vv[0].u, g0d);
                descending = false;
                l = 1;
                continue;
            }
            const SmallLevel<T> &L = S.lv[l];
            const SmallLevel<T> &C = S.lv[l - 1];
            const LevelVecs<T> V = vv[l];
            if (zero) {
                blk_fill(tm, V.u, 2 * L.n_int);
                tm.sync();
            }
            for (int j = 0; j < mlev[l]; ++j) blk_sweep(tm, L, V.g, V.u, false, rs);
            blk_residual(tm, L, V.g, V.u, V.r);
            blk_restrict(tm, L, C, V.r, vv[l - 1].g, V.c1, V.c2);
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
            const LevelVecs<T> V = vv[l];
            blk_prolong_add(tm, L, C, vv[l - 1].u, V.u, V.t);
            for (int j = 0; j < mlev[l]; ++j) blk_sweep(tm, L, V.g, V.u, true, rs);
            if (l == top) break;
            l = l + 1;
        }
    }
}

// carve the vectors of levels 0..top out of shared memory from `base` on, in the order
// the host sized them (mg_small_vec_bytes)
template <class T>
__device__ double *carve_levels(const SmallParams<T> &S, int top, unsigned char *base, LevelVecs<T> *vv) {
    for (int i = 0; i <= top; ++i) {
        const SmallLevel<T> &L = S.lv[i];
        const size_t n = 2 * (size_t)L.n_int;
        T *b = reinterpret_cast<T *>(base);
        vv[i] = LevelVecs<T>{b, b + n, b + 2 * n, b + 3 * n, b + 4 * n, b + 4 * n + 12 * (size_t)L.ncc};
        base += sizeof(T) * (4 * n + 18 * (size_t)L.ncc);
    }
    const size_t off = (reinterpret_cast<size_t>(base) + 7) & ~size_t(7);
    return reinterpret_cast<double *>(off);
}

template <class T, bool CL>
__global__ void __launch_bounds__(1024) mg_small_kernel(SmallParams<T> S, int l, int m, int zero_init) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ LevelVecs<T> vv[SMALL_MAX_LEVELS];
    __shared__ double *g0d;
    T *rs = reinterpret_cast<T *>(smraw);
    const Team<CL> tm = make_team<CL>();
    const bool resident = !CL && S.resident;
    if (threadIdx.x == 0) {
        if (resident) {
            g0d = carve_levels(S, l, smraw + S.vec_offset, vv);
        } else {
            for (int i = 0; i <= l; ++i) {
                const SmallLevel<T> &L = S.lv[i];
                vv[i] = LevelVecs<T>{L.g, L.u, L.r, L.t, L.ct1, L.ct2};
            }
            g0d = S.g0d;
        }
    }
    __syncthreads();
    const int n = 2 * S.lv[l].n_int;
    if (resident) {
        // the caller's right-hand side (and initial guess) in, the result out at the end
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            vv[l].g[i] = S.lv[l].g[i];
            if (!zero_init) vv[l].u[i] = S.lv[l].u[i];
        }
        __syncthreads();
    }
    blk_mg(tm, S, vv, g0d, l, m, zero_init != 0, rs);
    if (resident)
        for (int i = threadIdx.x; i < n; i += blockDim.x) S.lv[l].u[i] = vv[l].u[i];
}

cudaLaunchConfig_t cluster_config(int csize, size_t smem, cudaStream_t s, cudaLaunchAttribute &at) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(csize);
    cfg.blockDim = dim3(1024);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = csize;
    at.val.clusterDim.y = 1;
    at.val.clusterDim.z = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    return cfg;
}

} // namespace

// shared memory of the level vectors of levels 0..Ls kept resident by a single block
// (the layout carve_levels walks), including the FP64 coarse right-hand side
template <class T>
size_t mg_small_vec_bytes(const SmallParams<T> &S, int Ls) {
    size_t b = 0;
    for (int i = 0; i <= Ls; ++i) b += sizeof(T) * (8 * (size_t)S.lv[i].n_int + 18 * (size_t)S.lv[i].ncc);
    return b + 8 + sizeof(double) * 2 * (size_t)S.lv[0].n_int;
}

// shared memory per CTA when the largest colour phase (colour_bytes of residual
// rows) is split over csize CTAs; slack covers the rounding to whole patches
size_t mg_small_smem(size_t colour_bytes, int csize, int np_max_bytes) {
    return (colour_bytes + csize - 1) / csize + (size_t)np_max_bytes + 16;
}

// largest cluster (16, 8, 4, 2 CTAs of 1024 threads) this device can run with the
// shared memory of that split, or 1 (a single block); 0 if even one block does not fit
template <class T>
int mg_small_cluster_size(size_t colour_bytes, int np_max_bytes) {
    // a colour phase that one block covers in a single pass runs on one SM: no L2 round
    // trips and block barriers only
    if (colour_bytes / sizeof(T) <= 1024 && mg_small_smem(colour_bytes, 1, np_max_bytes) <= 200 * 1024) return 1;
    if (cudaFuncSetAttribute(mg_small_kernel<T, true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
        cudaGetLastError();
    for (int want : {16, 8, 4, 2}) {
        const size_t smem = mg_small_smem(colour_bytes, want, np_max_bytes);
        if (smem > 200 * 1024) continue;
        if (cudaFuncSetAttribute(mg_small_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        cudaLaunchAttribute at;
        cudaLaunchConfig_t cfg = cluster_config(want, smem, nullptr, at);
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, mg_small_kernel<T, true>, &cfg) == cudaSuccess && n >= 1) return want;
        cudaGetLastError();
    }
    return mg_small_smem(colour_bytes, 1, np_max_bytes) <= 200 * 1024 ? 1 : 0;
}

template <class T>
cudaError_t launch_mg_small(const SmallParams<T> &S, int l, int m, bool zero_init, size_t smem, int csize,
                            cudaStream_t s) {
    note_launches(1);
    if (csize <= 1) {
        cudaError_t e = cudaFuncSetAttribute(mg_small_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        mg_small_kernel<T, false><<<1, 1024, smem, s>>>(S, l, m, zero_init ? 1 : 0);
        return cudaGetLastError();
    }
    cudaError_t e = cudaFuncSetAttribute(mg_small_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute at;
    cudaLaunchConfig_t cfg = cluster_config(csize, smem, s, at);
    return cudaLaunchKernelEx(&cfg, mg_small_kernel<T, true>, S, l, m, zero_init ? 1 : 0);
}

template size_t mg_small_vec_bytes<double>(const SmallParams<double> &, int);
template size_t mg_small_vec_bytes<float>(const SmallParams<float> &, int);
template int mg_small_cluster_size<double>(size_t, int);
template int mg_small_cluster_size<float>(size_t, int);
template cudaError_t launch_mg_small<double>(const SmallParams<double> &, int, int, bool, size_t, int, cudaStream_t);
template cudaError_t launch_mg_small<float>(const SmallParams<float> &, int, int, bool, size_t, int, cudaStream_t);

} // namespace hdg
