// Hot-path kernels of the 3D path: four faces per cell, three lowest-order unknowns per face.
//
//  * apply3_kernel: y = A^eps x (or g - A^eps x), one thread per skeleton unknown, pulling the
//    rows of its face's two cells (Section 3.2 operator, condensed element matrices);
//  * gs3_kernel: one colour phase of block Gauss-Seidel over edge patches (Section 3.4.2 with
//    edges in place of vertices; eq. bjac's subspaces, relaxed multiplicatively): per patch the
//    star cells' unknowns are staged in shared memory, the patch residual formed from the two
//    cells of each patch face and the update applied through the transposed patch inverse;
//  * transfers between lowest-order levels (eqs. avgOpt, div-transfer, harmonic-ex): the
//    averaging of each fine face on a coarse face from its two coarse cells, the discrete
//    harmonic extension H = -A_TT^-1 A_TB per coarse cell, and the transposes;
//  * Π_k^0 / Π_0^k (Algorithm 2): the constant normal, t1 and t2 coefficients of each face.
#include <type_traits>

#include "hdg3d_internal.h"

namespace hdg {
namespace {

unsigned blocks_for(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

template <class T, int DPF>
__global__ void __launch_bounds__(256)
apply3_kernel(int64_t n_int, const int *__restrict__ facet_adj, const int *__restrict__ cell_int,
              const T *__restrict__ A, const T *__restrict__ x, const T *__restrict__ g, T *__restrict__ y) {
    constexpr int NLOC = 4 * DPF;
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n_int * DPF) return;
    const int64_t i = idx / DPF;
    const int d = (int)(idx - i * DPF);
    T acc = 0;
    for (int q = 0; q < 2; ++q) {
        const int adj = facet_adj[2 * i + q];
        if (adj < 0) continue;
        const int c = adj >> 2, lf = adj & 3;
        const T *Ac = A + (size_t)c * NLOC * NLOC + (size_t)lf * NLOC * DPF + d;
#pragma unroll
        for (int f2 = 0; f2 < 4; ++f2) {
            const int j = cell_int[4 * c + f2];
            if (j < 0) continue;
            const T *xs = x + (size_t)j * DPF;
#pragma unroll 6
            for (int d2 = 0; d2 < DPF; ++d2) acc += Ac[(f2 * DPF + d2) * DPF] * xs[d2];
        }
    }
    y[idx] = g ? g[idx] - acc : acc;
}

// One colour phase of the block GS over edge patches.  EXT (the FP64 sweep) takes the
// closed form: with P the patch's faces and E the two faces of each star cell without the
// patch edge, the update u_P <- u_P + A_PP^-1 (g - A u)_P equals A_PP^-1 (g_P - A_PE u_E),
// because Pinv is the inverse of the assembled A_PP; each (face, cell) slot then reads the two
// DPF x DPF coupling blocks of its face row with the cell's outside faces (contiguous in the
// row-block layout), half of the face's row block, and the patch overwrites u_P.  The FP32
// sweep keeps the correction form (whole row blocks): in FP32 the closed form applies the
// rounded inverse to O(gamma) values of the augmented-Lagrangian coupling, which costs a
// factor gamma of accuracy (the 2D sweeps split that term off; in 3D it is not split).
template <class T, int DPF, bool EXT>
__global__ void gs3_kernel(int p0, int p1, int pf_max, int pc_max, int np_max, const int *__restrict__ patch_nf,
                           const int *__restrict__ patch_facets, const int *__restrict__ patch_nc,
                           const int *__restrict__ patch_cells, const int *__restrict__ slot_src,
                           const int *__restrict__ cell_int, const int *__restrict__ patch_cext,
                           const T *__restrict__ A, const T *__restrict__ Pinv, const T *__restrict__ g,
                           T *__restrict__ u) {
    constexpr int NLOC = 4 * DPF;
    constexpr int NX = EXT ? 2 * DPF : NLOC;   // gathered unknowns per star cell
    extern __shared__ __align__(16) unsigned char smraw[];
    T *xs = reinterpret_cast<T *>(smraw);     // pc_max * NX
    T *r = xs + pc_max * NX;                   // np_max
    const int p = p0 + blockIdx.x;
    if (p >= p1) return;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int nf = patch_nf[p], ncell = patch_nc[p], np = nf * DPF;
    for (int t = tid; t < ncell * NX; t += nt) {
        const int si = t / NX, l = t % NX;
        const int c = patch_cells[(size_t)p * pc_max + si];
        const int f = EXT ? patch_cext[((size_t)p * pc_max + si) * 2 + l / DPF] : l / DPF;
        const int j = cell_int[4 * c + f];
        xs[t] = j >= 0 ? u[(size_t)j * DPF + l % DPF] : T(0);
    }
    __syncthreads();
    for (int t = tid; t < np; t += nt) {
        const int js = t / DPF, d = t % DPF;
        const int F = patch_facets[(size_t)p * pf_max + js];
        T acc = g[(size_t)F * DPF + d];
        for (int q = 0; q < 2; ++q) {
            const int src = slot_src[((size_t)p * pf_max + js) * 2 + q];
            const int si = src >> 2, lf = src & 3;
            const int c = patch_cells[(size_t)p * pc_max + si];
            const T *Ar = A + (size_t)c * NLOC * NLOC + (size_t)lf * NLOC * DPF + d;
            const T *xc = xs + si * NX;
            if constexpr (EXT) {
                for (int w = 0; w < 2; ++w) {
                    const T *Ac = Ar + (size_t)patch_cext[((size_t)p * pc_max + si) * 2 + w] * DPF * DPF;
#pragma unroll 6
                    for (int col = 0; col < DPF; ++col) acc -= Ac[col * DPF] * xc[w * DPF + col];
                }
            } else {
                for (int col = 0; col < NLOC; ++col) acc -= Ar[col * DPF] * xc[col];
            }
        }
        r[t] = acc;
    }
    __syncthreads();
    const T *Pi = Pinv + (size_t)p * np_max * np_max;
    for (int t = tid; t < np; t += nt) {
        T a0 = 0, a1 = 0;
        int j = 0;
        for (; j + 2 <= np; j += 2) {
            a0 += Pi[(size_t)j * np_max + t] * r[j];
            a1 += Pi[(size_t)(j + 1) * np_max + t] * r[j + 1];
        }
        if (j < np) a0 += Pi[(size_t)j * np_max + t] * r[j];
        const int F = patch_facets[(size_t)p * pf_max + t / DPF];
        if constexpr (EXT) u[(size_t)F * DPF + t % DPF] = a0 + a1;
        else u[(size_t)F * DPF + t % DPF] += a0 + a1;
    }
}

// prolongation, step 1: every fine face on a coarse interior face gets the mean of its two
// coarse cells' Π^CR values (W holds the 1/2), kept in tmp and added to uf
template <class T>
__global__ void prolong3_B_kernel(int64_t nB, const int *__restrict__ fineB, const int *__restrict__ fineB_src,
                                  const int *__restrict__ ccell_int, const T *__restrict__ W,
                                  const T *__restrict__ uc, T *__restrict__ tmp, T *__restrict__ uf) {
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nB) return;
    T v[3] = {0, 0, 0};
    for (int q = 0; q < 2; ++q) {
        const int src = fineB_src[2 * b + q];
        const int P = src >> 5, s = src & 31;
        const T *Wk = W + ((size_t)P * TR3_B + s) * 36;
        for (int cf = 0; cf < 4; ++cf) {
            const int j = ccell_int[4 * P + cf];
            if (j < 0) continue;
            for (int a2 = 0; a2 < 3; ++a2) {
                const T x = uc[3 * (size_t)j + a2];
                for (int a = 0; a < 3; ++a) v[a] += Wk[a * 12 + 3 * cf + a2] * x;
            }
        }
    }
    const int i = fineB[b];
    for (int a = 0; a < 3; ++a) {
        tmp[3 * (size_t)i + a] = v[a];
        uf[3 * (size_t)i + a] += v[a];
    }
}

// prolongation, step 2: the faces inside each coarse cell by the harmonic extension of its
// B values, u_T = H u_B
template <class T>
__global__ void prolong3_T_kernel(int64_t ncc, const int *__restrict__ slots, const T *__restrict__ H,
                                  const T *__restrict__ tmp, T *__restrict__ uf) {
    const int64_t P = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (P >= ncc) return;
    T b[3 * TR3_B];
    for (int s = 0; s < TR3_B; ++s) {
        const int i = slots[TR3_SLOTS * P + s];
        for (int a = 0; a < 3; ++a) b[3 * s + a] = i >= 0 ? tmp[3 * (size_t)i + a] : T(0);
    }
    const T *Hk = H + (size_t)P * (3 * TR3_T) * (3 * TR3_B);
    for (int t = 0; t < 3 * TR3_T; ++t) {
        T acc = 0;
        for (int c = 0; c < 3 * TR3_B; ++c) acc += Hk[t * 3 * TR3_B + c] * b[c];
        const int i = slots[TR3_SLOTS * P + TR3_B + t / 3];
        uf[3 * (size_t)i + t % 3] += acc;
    }
}

// restriction (the transpose), step 1: t1 = H^T r_T per coarse cell
template <class T>
__global__ void restrict3_T_kernel(int64_t ncc, const int *__restrict__ slots, const T *__restrict__ H,
                                   const T *__restrict__ rf, T *__restrict__ t1) {
    const int64_t P = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (P >= ncc) return;
    T rT[3 * TR3_T];
    for (int t = 0; t < 3 * TR3_T; ++t) rT[t] = rf[3 * (size_t)slots[TR3_SLOTS * P + TR3_B + t / 3] + t % 3];
    const T *Hk = H + (size_t)P * (3 * TR3_T) * (3 * TR3_B);
    for (int c = 0; c < 3 * TR3_B; ++c) {
        T acc = 0;
        for (int t = 0; t < 3 * TR3_T; ++t) acc += Hk[t * 3 * TR3_B + c] * rT[t];
        t1[(size_t)3 * TR3_B * P + c] = acc;
    }
}

// step 2: per coarse cell, W^T applied to the B faces' totals (fine residual plus both coarse
// cells' harmonic-extension terms)
template <class T>
__global__ void restrict3_B_kernel(int64_t ncc, const int *__restrict__ slots, const int *__restrict__ nbr,
                                   const T *__restrict__ W, const T *__restrict__ rf, const T *__restrict__ t1,
                                   T *__restrict__ t2) {
    const int64_t P = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (P >= ncc) return;
    T z[3 * TR3_B];
    for (int s = 0; s < TR3_B; ++s) {
        const int i = slots[TR3_SLOTS * P + s];
        if (i < 0) {
            z[3 * s] = z[3 * s + 1] = z[3 * s + 2] = 0;
            continue;
        }
        const int nb = nbr[TR3_B * P + s];
        const int Q = nb >> 5, s2 = nb & 31;
        for (int a = 0; a < 3; ++a)
            z[3 * s + a] = rf[3 * (size_t)i + a] + t1[(size_t)3 * TR3_B * P + 3 * s + a] +
                           t1[(size_t)3 * TR3_B * Q + 3 * s2 + a];
    }
    const T *Wk = W + (size_t)P * TR3_B * 36;
    for (int col = 0; col < 12; ++col) {
        T acc = 0;
        for (int row = 0; row < 3 * TR3_B; ++row) acc += Wk[row * 12 + col] * z[row];
        t2[12 * P + col] = acc;
    }
}

// step 3: each coarse interior face sums the contributions of its two cells
template <class T>
__global__ void restrict3_C_kernel(int64_t n_int_c, const int *__restrict__ facet_adj_c, const T *__restrict__ t2,
                                   T *__restrict__ rc) {
    const int64_t G = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (G >= n_int_c) return;
    T a[3] = {0, 0, 0};
    for (int q = 0; q < 2; ++q) {
        const int adj = facet_adj_c[2 * G + q];
        const int K = adj >> 2, lf = adj & 3;
        for (int b = 0; b < 3; ++b) a[b] += t2[12 * (size_t)K + 3 * lf + b];
    }
    for (int b = 0; b < 3; ++b) rc[3 * G + b] = a[b];
}

template <class T>
__global__ void hp3_restrict_kernel(int nf, int64_t n_int, const T *r, T *r0) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_int) return;
    for (int a = 0; a < 3; ++a) r0[3 * i + a] = r[i * 3 * nf + a * nf];
}

template <class T>
__global__ void hp3_prolong_kernel(int nf, int64_t n_int, const T *d0, T *u) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_int) return;
    for (int a = 0; a < 3; ++a) u[i * 3 * nf + a * nf] += d0[3 * i + a];
}

template <class T, int DPF>
cudaError_t apply3_launch(const DevLevel &L, const T *A, const T *x, const T *g, T *y, cudaStream_t s) {
    const int64_t n = L.n_int * DPF;
    if (n == 0) return cudaSuccess;
    note_launches(1);
    apply3_kernel<T, DPF><<<blocks_for(n, 256), 256, 0, s>>>(L.n_int, L.facet_adj.p, L.cell_int.p, A, x, g, y);
    return cudaGetLastError();
}

template <class T, int DPF>
cudaError_t gs3_launch(const DevLevel &L, const DevOperator &op, const T *A, const T *Pinv, int colour, const T *g,
                       T *u, cudaStream_t s) {
    const int p0 = L.colour_ptr[colour], p1 = L.colour_ptr[colour + 1];
    if (p1 <= p0) return cudaSuccess;
    int nt = ((op.np_max + 31) / 32) * 32;
    nt = std::min(std::max(nt, 32), 256);
    note_launches(1);
    if (std::is_same<T, double>::value && L.patch_cext.p) {
        const size_t smem = sizeof(T) * ((size_t)L.pc_max * 2 * DPF + op.np_max);
        gs3_kernel<T, DPF, true><<<p1 - p0, nt, smem, s>>>(p0, p1, L.pf_max, L.pc_max, op.np_max, L.patch_nf.p,
                                                           L.patch_facets.p, L.patch_nc.p, L.patch_cells.p,
                                                           L.patch_slot_src.p, L.cell_int.p, L.patch_cext.p, A,
                                                           Pinv, g, u);
    } else {
        const size_t smem = sizeof(T) * ((size_t)L.pc_max * 4 * DPF + op.np_max);
        gs3_kernel<T, DPF, false><<<p1 - p0, nt, smem, s>>>(p0, p1, L.pf_max, L.pc_max, op.np_max, L.patch_nf.p,
                                                            L.patch_facets.p, L.patch_nc.p, L.patch_cells.p,
                                                            L.patch_slot_src.p, L.cell_int.p, nullptr, A, Pinv, g,
                                                            u);
    }
    return cudaGetLastError();
}

} // namespace

template <class T>
cudaError_t launch_apply3(const DevLevel &L, int dpf, const T *A, const T *x, const T *g, T *y, cudaStream_t s) {
    switch (dpf) {
    case 3: return apply3_launch<T, 3>(L, A, x, g, y, s);
    case 9: return apply3_launch<T, 9>(L, A, x, g, y, s);
    case 18: return apply3_launch<T, 18>(L, A, x, g, y, s);
    case 30: return apply3_launch<T, 30>(L, A, x, g, y, s);
    default: return cudaErrorInvalidValue;
    }
}

template <class T>
cudaError_t launch_gs_colour3(const DevLevel &L, const DevOperator &op, const T *A, const T *Pinv, int colour,
                              const T *g, T *u, cudaStream_t s) {
    switch (op.dpf) {
    case 3: return gs3_launch<T, 3>(L, op, A, Pinv, colour, g, u, s);
    case 9: return gs3_launch<T, 9>(L, op, A, Pinv, colour, g, u, s);
    case 18: return gs3_launch<T, 18>(L, op, A, Pinv, colour, g, u, s);
    case 30: return gs3_launch<T, 30>(L, op, A, Pinv, colour, g, u, s);
    default: return cudaErrorInvalidValue;
    }
}

template <class T>
cudaError_t launch_prolong_add3(const DevLevel &F, const DevLevel &C, const T *W, const T *Hm, const T *uc, T *tmp,
                                T *uf, cudaStream_t s) {
    if (F.nB > 0) {
        note_launches(1);
        prolong3_B_kernel<T><<<blocks_for(F.nB, 128), 128, 0, s>>>(F.nB, F.tr_fineB.p, F.tr_fineB_src.p,
                                                                    C.cell_int.p, W, uc, tmp, uf);
    }
    if (F.nc_coarse > 0) {
        note_launches(1);
        prolong3_T_kernel<T><<<blocks_for(F.nc_coarse, 128), 128, 0, s>>>(F.nc_coarse, F.tr_slots.p, Hm, tmp, uf);
    }
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_restrict3(const DevLevel &F, const DevLevel &C, const T *W, const T *Hm, const T *rf, T *t1,
                             T *t2, T *rc, cudaStream_t s) {
    if (F.nc_coarse > 0) {
        note_launches(2);
        restrict3_T_kernel<T><<<blocks_for(F.nc_coarse, 128), 128, 0, s>>>(F.nc_coarse, F.tr_slots.p, Hm, rf, t1);
        restrict3_B_kernel<T><<<blocks_for(F.nc_coarse, 128), 128, 0, s>>>(F.nc_coarse, F.tr_slots.p, F.tr_nbr.p,
                                                                            W, rf, t1, t2);
    }
    if (C.n_int > 0) {
        note_launches(1);
        restrict3_C_kernel<T><<<blocks_for(C.n_int, 128), 128, 0, s>>>(C.n_int, C.facet_adj.p, t2, rc);
    }
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_hp_restrict3(int k, int64_t n_int, const T *r, T *r0, cudaStream_t s) {
    if (n_int == 0) return cudaSuccess;
    note_launches(1);
    hp3_restrict_kernel<T><<<blocks_for(n_int, 256), 256, 0, s>>>(nface3(k), n_int, r, r0);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_hp_prolong_add3(int k, int64_t n_int, const T *d0, T *u, cudaStream_t s) {
    if (n_int == 0) return cudaSuccess;
    note_launches(1);
    hp3_prolong_kernel<T><<<blocks_for(n_int, 256), 256, 0, s>>>(nface3(k), n_int, d0, u);
    return cudaGetLastError();
}

#define HDG_INST3(T)                                                                                               \
    template cudaError_t launch_apply3<T>(const DevLevel &, int, const T *, const T *, const T *, T *, cudaStream_t); \
    template cudaError_t launch_gs_colour3<T>(const DevLevel &, const DevOperator &, const T *, const T *, int,       \
                                              const T *, T *, cudaStream_t);                                        \
    template cudaError_t launch_prolong_add3<T>(const DevLevel &, const DevLevel &, const T *, const T *, const T *, \
                                                T *, T *, cudaStream_t);                                            \
    template cudaError_t launch_restrict3<T>(const DevLevel &, const DevLevel &, const T *, const T *, const T *,    \
                                             T *, T *, T *, cudaStream_t);                                          \
    template cudaError_t launch_hp_restrict3<T>(int, int64_t, const T *, T *, cudaStream_t);                       \
    template cudaError_t launch_hp_prolong_add3<T>(int, int64_t, const T *, T *, cudaStream_t);
HDG_INST3(double)
HDG_INST3(float)
#undef HDG_INST3

} // namespace hdg
