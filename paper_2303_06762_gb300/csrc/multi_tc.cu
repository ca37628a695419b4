// Batched order-k block Gauss-Seidel (Section 3.5, Algorithm 2 with R right-hand
// sides) on tensor cores: one colour phase, one CTA per vertex patch, for dpf = 8
// (k = 3) and R = 16, 32 or 64 columns, used by the batched preconditioner in
// the HDG_MIXED_FP16 / HDG_MIXED_BF16 precisions.
//
// Per patch both products of the block GS step are small dense GEMMs over the R
// columns, written transposed so that the R columns are the M dimension of
// mma.sync (m16n8k16 / m16n8k8, 16-bit operands, FP32 accumulation):
//   residual     Rsᵀ[r][(js,d)] = gᵀ - Σ_q  Xᵀ_{cell(js,q)}[r][0..24) · A_{js,q}[0..24)[d]
//   block solve  Δuᵀ[r][n]      = Σ_j Rsᵀ[r][j] · (A_ss⁻¹)ᵀ[j][n]
// A_{js,q} is the facet row block of the (js, q) slot's element matrix, read from
// the 16-bit row-scaled copy (row scales applied to the FP32 accumulators); the
// inverse likewise.  The gathered unknowns X and the residual are rounded to the
// 16-bit format per column r with a power-of-two scale (largest magnitude of the
// column over the patch in [1/2, 1)), so that every column's result depends on
// that column only.  Operand fragments come from shared memory by ldmatrix.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "hdg_internal.h"

namespace hdg {
namespace {

constexpr int TC_DPF = 8;
constexpr int TC_NLOC = 3 * TC_DPF;
constexpr int TC_XS = TC_NLOC;   // 16-bit values per Xᵀ row (48-byte rows: conflict-free ldmatrix)

template <class H>
struct Mma;

template <>
struct Mma<__half> {
    static __device__ __forceinline__ void k16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
        asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                     "{%0,%1,%2,%3};"
                     : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                     : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
    static __device__ __forceinline__ void k8(float (&c)[4], const uint32_t (&a)[2], uint32_t b) {
        asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
                     "{%0,%1,%2,%3};"
                     : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                     : "r"(a[0]), "r"(a[1]), "r"(b));
    }
    static __device__ __forceinline__ __half from(float v) { return __float2half_rn(v); }
};

template <>
struct Mma<__nv_bfloat16> {
    static __device__ __forceinline__ void k16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
        asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                     "{%0,%1,%2,%3};"
                     : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                     : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
    static __device__ __forceinline__ void k8(float (&c)[4], const uint32_t (&a)[2], uint32_t b) {
        asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
                     "{%0,%1,%2,%3};"
                     : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                     : "r"(a[0]), "r"(a[1]), "r"(b));
    }
    static __device__ __forceinline__ __nv_bfloat16 from(float v) { return __float2bfloat16_rn(v); }
};

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// 8x8 16-bit matrices from shared memory: lanes 8i..8i+7 give the row addresses of matrix i
__device__ __forceinline__ void ldm_x4(uint32_t (&r)[4], uint32_t a) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(a) : "memory");
}
__device__ __forceinline__ void ldm_x2(uint32_t (&r)[2], uint32_t a) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(a) : "memory");
}
__device__ __forceinline__ void ldm_x2_t(uint32_t (&r)[2], uint32_t a) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];"
                 : "=r"(r[0]), "=r"(r[1]) : "r"(a) : "memory");
}
__device__ __forceinline__ void ldm_x1_t(uint32_t &r, uint32_t a) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x1.trans.shared.b16 {%0}, [%1];" : "=r"(r) : "r"(a) : "memory");
}

// power-of-two scale of a column whose largest magnitude has the bits `mx`: returns
// 1/s and sets s, with the largest scaled magnitude in [1/2, 1)
__device__ __forceinline__ float col_scale(unsigned mx, float &s) {
    const float m = __uint_as_float(mx);
    int e = 0;
    if (m > 0.f && isfinite(m)) frexpf(m, &e);
    s = ldexpf(1.f, e);
    return ldexpf(1.f, -e);
}

struct TcLayout {
    size_t xt, as, ps, rs, rf, asc, psc, cmx, rmx, xsc, rsc, roff, rowF, sslot, total;
};

// shared-memory layout (byte offsets, each a multiple of 16)
__host__ __device__ inline TcLayout tc_layout(int pf_max, int pc_max, int np_max, int R) {
    auto up = [](size_t b) { return (b + 15) & ~size_t(15); };
    const size_t psd = (size_t)np_max + 8;
    TcLayout o{};
    size_t at = 0;
    o.xt = at;   at = up(at + 2 * (size_t)pc_max * R * TC_XS);
    o.as = at;   at = up(at + 2 * (size_t)2 * pf_max * TC_NLOC * TC_DPF);
    o.ps = at;   at = up(at + 2 * (size_t)np_max * psd);
    o.rs = at;   at = up(at + 2 * (size_t)R * psd);
    o.rf = at;   at = up(at + 4 * (size_t)np_max * R);
    o.asc = at;  at = up(at + 4 * (size_t)2 * pf_max * TC_DPF);
    o.psc = at;  at = up(at + 4 * (size_t)np_max);
    o.cmx = at;  at = up(at + 4 * (size_t)R);
    o.rmx = at;  at = up(at + 4 * (size_t)R);
    o.xsc = at;  at = up(at + 4 * (size_t)2 * R);
    o.rsc = at;  at = up(at + 4 * (size_t)2 * R);
    o.roff = at; at = up(at + 4 * (size_t)pc_max * TC_NLOC);
    o.rowF = at; at = up(at + 4 * (size_t)pf_max);
    o.sslot = at; at = up(at + 4 * (size_t)2 * pf_max);
    o.total = at;
    return o;
}

// NT: threads per block (128 or 256, chosen by the autotuner); a multiple of R, so that each
// thread's column r = tid mod R stays fixed in the column-maximum pass
template <class H, int NT>
__global__ void __launch_bounds__(NT)
gs_tc_kernel(int p0, int p1, int pf_max, int pc_max, int np_max, int lgR, const int *__restrict__ patch_nf,
             const int *__restrict__ patch_facets, const int *__restrict__ patch_nc,
             const int *__restrict__ patch_cells, const int *__restrict__ slot_src,
             const int *__restrict__ cell_int, const H *__restrict__ Ah, const float *__restrict__ Ah_s,
             const H *__restrict__ Ph, const float *__restrict__ Ph_s, const float *__restrict__ g,
             float *__restrict__ u) {
    constexpr int DPF = TC_DPF, NLOC = TC_NLOC, RBK = NLOC * DPF;
    const int R = 1 << lgR, psd = np_max + 8;
    extern __shared__ __align__(16) unsigned char smraw[];
    const TcLayout L = tc_layout(pf_max, pc_max, np_max, R);
    H *XT = reinterpret_cast<H *>(smraw + L.xt);        // [star cell][r][col]
    H *AS = reinterpret_cast<H *>(smraw + L.as);        // [slot][col][d]
    H *PS = reinterpret_cast<H *>(smraw + L.ps);        // [j][n], row stride psd
    H *RS = reinterpret_cast<H *>(smraw + L.rs);        // [r][j], row stride psd
    float *RF = reinterpret_cast<float *>(smraw + L.rf);  // [j][r] FP32 residual
    float *asc = reinterpret_cast<float *>(smraw + L.asc);
    float *psc = reinterpret_cast<float *>(smraw + L.psc);
    unsigned *cmx = reinterpret_cast<unsigned *>(smraw + L.cmx);
    unsigned *rmx = reinterpret_cast<unsigned *>(smraw + L.rmx);
    float *xsc = reinterpret_cast<float *>(smraw + L.xsc);   // [r]: scale, [R + r]: its inverse
    float *rsc = reinterpret_cast<float *>(smraw + L.rsc);
    int *roff = reinterpret_cast<int *>(smraw + L.roff);     // star slot -> first row of u, or -1
    int *rowF = reinterpret_cast<int *>(smraw + L.rowF);
    int *sslot = reinterpret_cast<int *>(smraw + L.sslot);

    const int p = p0 + blockIdx.x;
    if (p >= p1) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = NT / 32;
    const int nf = patch_nf[p], ncell = patch_nc[p], np = nf * DPF;

    for (int i = tid; i < ncell * NLOC; i += NT) {
        const int si = i / NLOC, l = i - si * NLOC;
        const int c = patch_cells[(size_t)p * pc_max + si];
        const int j = cell_int[3 * c + l / DPF];
        roff[i] = j >= 0 ? (j * DPF + l % DPF) << lgR : -1;
    }
    for (int i = tid; i < R; i += NT) cmx[i] = rmx[i] = 0u;
    for (int js = tid; js < nf; js += NT) rowF[js] = patch_facets[(size_t)p * pf_max + js];
    for (int sl = tid; sl < 2 * nf; sl += NT) sslot[sl] = slot_src[(size_t)p * pf_max * 2 + sl] >> 2;
    // facet row blocks of the 2 nf slots (slot js*2 + q), 16-byte vectors
    constexpr int VB = RBK * 2 / 16;
    for (int i = tid; i < 2 * nf * VB; i += NT) {
        const int sl = i / VB, v = i - sl * VB;
        const int src = slot_src[(size_t)p * pf_max * 2 + sl];
        const int c = patch_cells[(size_t)p * pc_max + (src >> 2)];
        reinterpret_cast<uint4 *>(AS + (size_t)sl * RBK)[v] =
            reinterpret_cast<const uint4 *>(Ah + (size_t)c * NLOC * NLOC + (size_t)(src & 3) * RBK)[v];
    }
    for (int i = tid; i < 2 * nf * DPF; i += NT) {
        const int sl = i / DPF, d = i - sl * DPF;
        const int src = slot_src[(size_t)p * pf_max * 2 + sl];
        const int c = patch_cells[(size_t)p * pc_max + (src >> 2)];
        asc[i] = Ah_s[(size_t)c * NLOC + (src & 3) * DPF + d];
    }
    // the inverse's rows j < np (np_max values each, stored transposed: [j][n] = (A_ss⁻¹)_nj)
    const int pv = np_max / 8;
    for (int i = tid; i < np * pv; i += NT) {
        const int j = i / pv, v = i - j * pv;
        reinterpret_cast<uint4 *>(PS + (size_t)j * psd)[v] =
            reinterpret_cast<const uint4 *>(Ph + (size_t)p * np_max * np_max + (size_t)j * np_max)[v];
    }
    for (int i = tid; i < np; i += NT) psc[i] = Ph_s[(size_t)p * np_max + i];
    __syncthreads();

    // gathered unknowns of the star: column maxima (the thread's column is fixed, since
    // the block size is a multiple of R: one shared atomic per thread), per-column scales,
    // then the scaled 16-bit Xᵀ
    const int nx = (ncell * NLOC) << lgR;
    {
        float m = 0.f;
        for (int t = tid; t < nx; t += NT) {
            const int o = roff[t >> lgR];
            if (o >= 0) m = fmaxf(m, fabsf(u[o + (t & (R - 1))]));
        }
        atomicMax(&cmx[tid & (R - 1)], __float_as_uint(m));
    }
    __syncthreads();
    for (int r = tid; r < R; r += NT) {
        float sc;
        xsc[R + r] = col_scale(cmx[r], sc);
        xsc[r] = sc;
    }
    __syncthreads();
    for (int t = tid; t < nx; t += NT) {
        const int r = t & (R - 1), sl = t >> lgR, si = sl / NLOC, l = sl - si * NLOC;
        const int o = roff[sl];
        const float v = o >= 0 ? u[o + r] : 0.f;
        XT[((size_t)si * R + r) * TC_XS + l] = Mma<H>::from(v * xsc[R + r]);
    }
    __syncthreads();

    const int nrt = R >> 4, g8 = lane >> 2, t4 = lane & 3;
    const int arow = (lane & 7) + ((lane >> 3) & 1) * 8;   // ldmatrix row of this lane in a 16-row tile
    // residual: tile (rt, js) = 16 columns x the 8 rows of facet js
    for (int tile = warp; tile < nrt * nf; tile += NW) {
        const int rt = tile % nrt, js = tile / nrt;
        float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int sl = 2 * js + q, si = sslot[sl];
            const H *xrow = XT + ((size_t)si * R + rt * 16 + arow) * TC_XS;
            uint32_t a[4], b[2];
            ldm_x4(a, saddr(xrow + (lane >> 4) * 8));                          // columns 0..15
            ldm_x2_t(b, saddr(AS + ((size_t)sl * NLOC + (lane & 15)) * DPF));
            Mma<H>::k16(acc[q], a, b);
            uint32_t a2[2], b1;
            ldm_x2(a2, saddr(xrow + 16));                                      // columns 16..23
            ldm_x1_t(b1, saddr(AS + ((size_t)sl * NLOC + 16 + (lane & 7)) * DPF));
            Mma<H>::k8(acc[q], a2, b1);
        }
        const int F = rowF[js];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int r = rt * 16 + g8 + 8 * h;
            const float s = xsc[r];
            float m = 0.f;
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int d = 2 * t4 + e;
                const float prod = asc[(2 * js) * DPF + d] * acc[0][2 * h + e] +
                                   asc[(2 * js + 1) * DPF + d] * acc[1][2 * h + e];
                const float v = g[(((size_t)F * DPF + d) << lgR) + r] - s * prod;
                RF[(size_t)(js * DPF + d) * R + r] = v;
                m = fmaxf(m, fabsf(v));
            }
            // the four lanes of a quad hold the 8 rows of column r
            m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
            m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
            if (t4 == 0) atomicMax(&rmx[r], __float_as_uint(m));
        }
    }
    __syncthreads();
    for (int r = tid; r < R; r += NT) {
        float sc;
        rsc[R + r] = col_scale(rmx[r], sc);
        rsc[r] = sc;
    }
    __syncthreads();
    for (int t = tid; t < (np << lgR); t += NT) {
        const int j = t >> lgR, r = t & (R - 1);
        RS[(size_t)r * psd + j] = Mma<H>::from(RF[t] * rsc[R + r]);
    }
    __syncthreads();

    // block solve: tile (rt, nt) = 16 columns x 8 rows n of the patch
    const int nnt = np / 8;
    for (int tile = warp; tile < nrt * nnt; tile += NW) {
        const int rt = tile % nrt, nt = tile / nrt;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        const H *rrow = RS + (size_t)(rt * 16 + arow) * psd;
        int k0 = 0;
        for (; k0 + 16 <= np; k0 += 16) {
            uint32_t a[4], b[2];
            ldm_x4(a, saddr(rrow + k0 + (lane >> 4) * 8));
            ldm_x2_t(b, saddr(PS + (size_t)(k0 + (lane & 15)) * psd + nt * 8));
            Mma<H>::k16(acc, a, b);
        }
        if (k0 < np) {
            uint32_t a2[2], b1;
            ldm_x2(a2, saddr(rrow + k0));
            ldm_x1_t(b1, saddr(PS + (size_t)(k0 + (lane & 7)) * psd + nt * 8));
            Mma<H>::k8(acc, a2, b1);
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int r = rt * 16 + g8 + 8 * h;
            const float s = rsc[r];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int n = nt * 8 + 2 * t4 + e;
                u[(((size_t)rowF[n / DPF] * DPF + n % DPF) << lgR) + r] += s * psc[n] * acc[2 * h + e];
            }
        }
    }
}

template <class H, int NT>
cudaError_t gs_tc_launch(const DevLevel &L, const DevOperator &op, int R, int colour, const float *g, float *u,
                         cudaStream_t s) {
    const int p0 = L.colour_ptr[colour], p1 = L.colour_ptr[colour + 1];
    if (p1 <= p0) return cudaSuccess;
    const size_t smem = tc_layout(L.pf_max, L.pc_max, op.np_max, R).total;
    cudaError_t e = cudaFuncSetAttribute(gs_tc_kernel<H, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    note_launches(1);
    gs_tc_kernel<H, NT><<<p1 - p0, NT, smem, s>>>(
        p0, p1, L.pf_max, L.pc_max, op.np_max, log2_width(R), L.patch_nf.p, L.patch_facets.p, L.patch_nc.p,
        L.patch_cells.p, L.patch_slot_src.p, L.cell_int.p, reinterpret_cast<const H *>(op.Ah.p), op.Ah_s.p,
        reinterpret_cast<const H *>(op.Pinvh.p), op.Pinvh_s.p, g, u);
    return cudaGetLastError();
}

} // namespace

bool gs_tc_supported(const DevLevel &L, const DevOperator &op, int R) {
    if (op.h_fmt != HDG_MIXED_FP16 && op.h_fmt != HDG_MIXED_BF16) return false;
    if (op.dpf != TC_DPF || (R != 16 && R != 32 && R != 64) || op.np_max % 8 != 0) return false;
    return tc_layout(L.pf_max, L.pc_max, op.np_max, R).total <= 200 * 1024;
}

cudaError_t launch_gs_colour_tc(const DevLevel &L, const DevOperator &op, int R, int colour, const float *g,
                                float *u, cudaStream_t s, int nt) {
    if (!gs_tc_supported(L, op, R)) return cudaErrorInvalidValue;
    const bool bf = op.h_fmt == HDG_MIXED_BF16;
    if (nt == 128) return bf ? gs_tc_launch<__nv_bfloat16, 128>(L, op, R, colour, g, u, s)
                             : gs_tc_launch<__half, 128>(L, op, R, colour, g, u, s);
    if (nt != 0 && nt != 256) return cudaErrorInvalidValue;
    return bf ? gs_tc_launch<__nv_bfloat16, 256>(L, op, R, colour, g, u, s)
              : gs_tc_launch<__half, 256>(L, op, R, colour, g, u, s);
}

} // namespace hdg
