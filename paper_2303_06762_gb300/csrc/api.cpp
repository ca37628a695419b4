// C ABI of the GB300 H(div)-HDG hp-multigrid library: context management,
// setup (topology upload, condensation driver), and the host orchestration of
// the hot path: Algorithm 1 (MG_h), Algorithm 2 (MG_hp), flexible GMRES and the
// augmented-Lagrangian Uzawa iteration (eq. stOpEq-ALU).  Every numerical step
// runs in the CUDA kernels of condense.cu / ops.cu; this file only sequences
// launches on the caller's stream and reads back the few scalars that decide
// convergence.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "hdg3d_internal.h"

using namespace hdg;

namespace {

struct Fail {
    hdg_status st;
};

#define CK(expr)                                                                             \
    do {                                                                                     \
        cudaError_t e_ = (expr);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            ctx->err = std::string(#expr) + ": " + cudaGetErrorString(e_);                  \
            throw Fail{e_ == cudaErrorMemoryAllocation ? HDG_ERR_OOM : HDG_ERR_CUDA};        \
        }                                                                                    \
    } while (0)

#define REQUIRE(cond, msg)                                                                   \
    do {                                                                                     \
        if (!(cond)) {                                                                       \
            ctx->err = (msg);                                                                \
            throw Fail{HDG_ERR_INVALID_ARG};                                                 \
        }                                                                                    \
    } while (0)

template <class T>
void dalloc(hdg_ctx *ctx, DBuf<T> &b, size_t n) {
    if (b.p && b.n >= n) return;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.n = 0;
    if (n == 0) return;
    CK(cudaMalloc((void **)&b.p, sizeof(T) * n));
    b.n = n;
}

template <class T>
void dfree(DBuf<T> &b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.n = 0;
}

template <class T>
void upload(hdg_ctx *ctx, DBuf<T> &b, const std::vector<T> &h) {
    dalloc(ctx, b, h.size());
    if (!h.empty()) CK(cudaMemcpy(b.p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
}

void free_operator(DevOperator &op) {
    dfree(op.A);
    dfree(op.Af);
    dfree(op.Alo);
    dfree(op.Fel);
    dfree(op.Pinv);
    dfree(op.Pinvf);
    dfree(op.Pinvp);
    dfree(op.Ah);
    dfree(op.Ah_s);
    dfree(op.Pinvh);
    dfree(op.Pinvh_s);
    dfree(op.swQ);
    dfree(op.swA00);
    op.h_fmt = 0;
}

void free_level(DevLevel &L) {
    dfree(L.coords); dfree(L.cells); dfree(L.cell_int); dfree(L.facet_adj); dfree(L.cell_d); dfree(L.cell_nu);
    dfree(L.cell_area); dfree(L.conv_flux); dfree(L.conv_lat); dfree(L.patch_nf); dfree(L.patch_facets); dfree(L.patch_nc);
    dfree(L.patch_cells); dfree(L.patch_slot_src); dfree(L.gs0_table); dfree(L.facet_slot); dfree(L.cell_bnd); dfree(L.patch_cint);
    dfree(L.patch_cext);
    free_operator(L.op0);
    dfree(L.tr_slots); dfree(L.tr_nbr); dfree(L.tr_children); dfree(L.tr_child_slot);
    dfree(L.tr_fineB); dfree(L.tr_fineB_src); dfree(L.tr_W); dfree(L.tr_H); dfree(L.tr_Wf);
    dfree(L.tr_Hf);
    dfree(L.g); dfree(L.u); dfree(L.r); dfree(L.t);
    dfree(L.gf); dfree(L.uf); dfree(L.rf); dfree(L.tf);
    dfree(L.ct1); dfree(L.ct2); dfree(L.ct1f); dfree(L.ct2f);
    for (auto *b : {&L.mg, &L.mu, &L.mr, &L.mt, &L.mc1, &L.mc2}) dfree(*b);
    for (auto *b : {&L.mgf, &L.muf, &L.mrf, &L.mtf, &L.mc1f, &L.mc2f}) dfree(*b);
}

template <class Fn>
hdg_status guard(hdg_ctx *ctx, Fn &&fn) {
    try {
        fn();
        return HDG_OK;
    } catch (const Fail &f) {
        return f.st;
    } catch (const std::exception &e) {
        if (ctx) ctx->err = e.what();
        return HDG_ERR_INVALID_ARG;
    } catch (...) {
        if (ctx) ctx->err = "unknown exception";
        return HDG_ERR_CUDA;
    }
}

void check_flag(hdg_ctx *ctx, cudaStream_t s) {
    int flag = 0;
    CK(cudaMemcpyAsync(&flag, ctx->status_flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (flag) {
        ctx->err = "non-positive pivot in a factorisation (flag " + std::to_string(flag) + ")";
        throw Fail{HDG_ERR_SINGULAR};
    }
}

// a kernel gave up a bounded wait (the bulk copies of the order-k sweep): its update was
// skipped, so the result of the call is wrong; the flag is cleared for the next call
void check_wait_flag(hdg_ctx *ctx, cudaStream_t s) {
    int flag = 0;
    CK(cudaMemcpyAsync(&flag, ctx->wait_flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (flag) {
        CK(cudaMemsetAsync(ctx->wait_flag.p, 0, sizeof(int), s));
        ctx->err = "a device wait timed out (flag " + std::to_string(flag) + ")";
        throw Fail{HDG_ERR_TIMEOUT};
    }
}

// the same check for the step-level entry points that may run the bulk-copy sweep (the
// order-k FP32 smoother): skipped when that sweep cannot have run, or while the caller's
// stream is being captured (the capture owner checks at its own synchronisation point)
void check_wait_flag_sweep(hdg_ctx *ctx, cudaStream_t s) {
    if (!ctx->opk.tma_flag || ctx->prm.precision == HDG_FP64) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone) return;
    check_wait_flag(ctx, s);
}

double read_scalar(hdg_ctx *ctx, const double *dev, cudaStream_t s) {
    CK(cudaMemcpyAsync(ctx->h_pinned, dev, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return ctx->h_pinned[0];
}

// ---------------------------------------------------------------- MG_h (Algorithm 1)
template <class T>
struct Prec;

template <>
struct Prec<double> {
    static const double *A(const DevOperator &o) { return o.A.p; }
    static const double *P(const DevOperator &o) { return o.Pinv.p; }
    static double *g(DevLevel &L) { return L.g.p; }
    static double *u(DevLevel &L) { return L.u.p; }
    static double *r(DevLevel &L) { return L.r.p; }
    static double *t(DevLevel &L) { return L.t.p; }
    static double *c1(DevLevel &L) { return L.ct1.p; }
    static double *c2(DevLevel &L) { return L.ct2.p; }
    static const double *W(const DevLevel &L) { return L.tr_W.p; }
    static const double *H(const DevLevel &L) { return L.tr_H.p; }
};
template <>
struct Prec<float> {
    static const float *A(const DevOperator &o) { return o.Af.p; }
    static const float *P(const DevOperator &o) { return o.Pinvf.p; }
    static float *g(DevLevel &L) { return L.gf.p; }
    static float *u(DevLevel &L) { return L.uf.p; }
    static float *r(DevLevel &L) { return L.rf.p; }
    static float *t(DevLevel &L) { return L.tf.p; }
    static float *c1(DevLevel &L) { return L.ct1f.p; }
    static float *c2(DevLevel &L) { return L.ct2f.p; }
    static const float *W(const DevLevel &L) { return L.tr_Wf.p; }
    static const float *H(const DevLevel &L) { return L.tr_Hf.p; }
};

template <class T>
void apply_op(hdg_ctx *ctx, const DevLevel &L, const DevOperator &op, const T *x, const T *g, T *y,
              cudaStream_t s);

// one step of the damped block Jacobi smoother (eq. bjac): r = g - A u in the residual work
// vector of the level (the order-k one for the order-k operator), every patch's correction,
// then u += damping x (the two corrections of each unknown); forward = backward
template <class T>
void jacobi_step(hdg_ctx *ctx, const DevLevel &L, const DevOperator &op, const T *g, T *u, cudaStream_t s) {
    const bool dbl = std::is_same<T, double>::value;
    T *r = &op == &ctx->opk ? (dbl ? (T *)ctx->kr.p : (T *)ctx->krf.p) : Prec<T>::r(const_cast<DevLevel &>(L));
    T *D = dbl ? (T *)ctx->jD.p : (T *)ctx->jDf.p;
    apply_op<T>(ctx, L, op, u, g, r, s);
    const double damp = ctx->prm.jacobi_damping > 0 ? ctx->prm.jacobi_damping : 0.5;
    CK(launch_jacobi_update<T>(L, op, Prec<T>::P(op), r, D, damp, u, s));
}

// one sweep of block GS; FP32 sweeps of an operator with 16-bit copies read those
template <class T>
void sweep(hdg_ctx *ctx, const DevLevel &L, const DevOperator &op, const T *g, T *u, bool reverse,
           cudaStream_t s) {
    if (ctx->prm.smoother == 1) {
        jacobi_step<T>(ctx, L, op, g, u, s);
        return;
    }
    for (int i = 0; i < L.n_colours; ++i) {
        int c = reverse ? L.n_colours - 1 - i : i;
        if constexpr (std::is_same<T, float>::value) {
            if (op.h_fmt) {
                CK(launch_gs_colour_h(L, op, c, g, u, s));
                continue;
            }
        }
        CK(launch_gs_colour<T>(L, op, Prec<T>::A(op), Prec<T>::P(op), c, g, u, s));
    }
}

// y = A x (or g - A x) in the preconditioner's precision, likewise on the 16-bit copies
template <class T>
void apply_op(hdg_ctx *ctx, const DevLevel &L, const DevOperator &op, const T *x, const T *g, T *y,
              cudaStream_t s) {
    if constexpr (std::is_same<T, float>::value) {
        if (op.h_fmt) {
            CK(launch_apply_h(L, op, x, g, y, s));
            return;
        }
    }
    CK(launch_apply<T>(L, op, Prec<T>::A(op), x, g, y, s));
}

template <class T>
void coarse_solve(hdg_ctx *ctx, cudaStream_t s) {
    DevLevel &L0 = ctx->L[0];
    int64_t n = L0.dim * L0.n_int;
    if constexpr (std::is_same<T, double>::value) {
        CK(launch_coarse_apply(ctx->coarse_inv.p, n, L0.g.p, L0.u.p, s));
    } else {
        CK(launch_f2d(L0.gf.p, L0.g.p, n, s));
        CK(launch_coarse_apply(ctx->coarse_inv.p, n, L0.g.p, L0.u.p, s));
        CK(launch_d2f(L0.u.p, L0.uf.p, n, s));
    }
}

template <class T>
SmallParams<T> &small_of(hdg_ctx *ctx);
template <>
SmallParams<double> &small_of<double>(hdg_ctx *ctx) { return ctx->small_d; }
template <>
SmallParams<float> &small_of<float>(hdg_ctx *ctx) { return ctx->small_f; }

template <class T>
size_t fill_small(hdg_ctx *ctx, int Ls) {
    SmallParams<T> &S = small_of<T>(ctx);
    S = SmallParams<T>();
    S.inv = ctx->coarse_inv.p;
    S.g0d = ctx->L[0].g.p;
    S.q = ctx->prm.cycle;
    S.growth = ctx->prm.vcycle_growth;
    size_t smem = 0;
    for (int l = 0; l <= Ls; ++l) {
        DevLevel &L = ctx->L[l];
        SmallLevel<T> &V = S.lv[l];
        V.n_int = (int)L.n_int;
        V.n_colours = L.n_colours;
        V.pf_max = L.pf_max;
        V.pc_max = L.pc_max;
        V.np_max = L.op0.np_max;
        for (int c = 0; c <= L.n_colours; ++c) V.colour_ptr[c] = L.colour_ptr[c];
        V.cell_int = L.cell_int.p;
        V.facet_adj = L.facet_adj.p;
        V.patch_nf = L.patch_nf.p;
        V.patch_facets = L.patch_facets.p;
        V.patch_cells = L.patch_cells.p;
        V.slot_src = L.patch_slot_src.p;
        V.A = Prec<T>::A(L.op0);
        V.Pinv = Prec<T>::P(L.op0);
        V.g = Prec<T>::g(L);
        V.u = Prec<T>::u(L);
        V.r = Prec<T>::r(L);
        V.t = Prec<T>::t(L);
        if (l > 0) {
            V.ncc = (int)L.nc_coarse;
            V.nB = (int)L.nB;
            V.tr_slots = L.tr_slots.p;
            V.tr_nbr = L.tr_nbr.p;
            V.tr_fineB = L.tr_fineB.p;
            V.tr_fineB_src = L.tr_fineB_src.p;
            V.W = Prec<T>::W(L);
            V.H = Prec<T>::H(L);
            V.ct1 = Prec<T>::c1(L);
            V.ct2 = Prec<T>::c2(L);
            for (int c = 0; c < L.n_colours; ++c)
                smem = std::max(smem, (size_t)(L.colour_ptr[c + 1] - L.colour_ptr[c]) * L.op0.np_max * sizeof(T));
        }
    }
    return std::max<size_t>(smem, 16);
}

template <class T>
void make_resident(SmallParams<T> &S, int Ls, size_t &smem) {
    const size_t off = (smem + 15) & ~size_t(15);
    const size_t vb = mg_small_vec_bytes(S, Ls);
    if (off + vb > 200 * 1024) return;
    S.resident = 1;
    S.vec_offset = off;
    smem = off + vb;
}

// largest level Ls >= 1 whose levels 0..Ls all fit the single-block kernel, else -1
int small_levels(hdg_ctx *ctx) {
    int Ls = -1;
    for (int l = 0; l < std::min(ctx->n_levels, SMALL_MAX_LEVELS); ++l) {
        const DevLevel &L = ctx->L[l];
        if (L.nc > ctx->prm.fused_coarse_cells || L.nc > SMALL_MAX_CELLS ||
            L.n_colours > SMALL_MAX_COLOURS)
            break;
        Ls = l;
    }
    return Ls >= 1 ? Ls : -1;
}

// u_l = MG_h(l, g_l, u_l (zero_init ? 0 : as is), m, q)
template <class T>
void mg_h(hdg_ctx *ctx, int l, int m, bool zero_init, cudaStream_t s) {
    if (l >= 1 && l <= ctx->small_Ls) {
        const bool dbl = std::is_same<T, double>::value;
        CK(launch_mg_small<T>(small_of<T>(ctx), l, m, zero_init, dbl ? ctx->small_smem_d : ctx->small_smem_f,
                              dbl ? ctx->small_cs_d : ctx->small_cs_f, s));
        return;
    }
    if (l == 0) {
        coarse_solve<T>(ctx, s);
        return;
    }
    DevLevel &L = ctx->L[l];
    DevLevel &C = ctx->L[l - 1];
    const int64_t n = L.dim * L.n_int;
    T *g = Prec<T>::g(L), *u = Prec<T>::u(L), *r = Prec<T>::r(L);
    if (zero_init) CK(launch_fill<T>(u, T(0), n, s));
    for (int j = 0; j < m; ++j) sweep<T>(ctx, L, L.op0, g, u, false, s);
    CK(launch_apply<T>(L, L.op0, Prec<T>::A(L.op0), u, g, r, s));
    CK(launch_restrict<T>(L, C, Prec<T>::W(L), Prec<T>::H(L), r, Prec<T>::c1(L), Prec<T>::c2(L),
                          Prec<T>::g(C), s));
    const int q = ctx->prm.cycle;
    const int mc = (q == 1) ? m * ctx->prm.vcycle_growth : m;
    for (int it = 0; it < q; ++it) mg_h<T>(ctx, l - 1, mc, it == 0, s);
    CK(launch_prolong_add<T>(L, C, Prec<T>::W(L), Prec<T>::H(L), Prec<T>::u(C), Prec<T>::t(L), u, s));
    for (int j = 0; j < m; ++j) sweep<T>(ctx, L, L.op0, g, u, true, s);
}

// Π_k^0 and Π_0^k of the level's dimension
template <class T>
cudaError_t hp_restrict_any(const DevLevel &L, int k, const T *r, T *r0, cudaStream_t s) {
    return L.dim == 3 ? launch_hp_restrict3<T>(k, L.n_int, r, r0, s) : launch_hp_restrict<T>(k, L.n_int, r, r0, s);
}
template <class T>
cudaError_t hp_prolong_any(const DevLevel &L, int k, const T *d0, T *u, cudaStream_t s) {
    return L.dim == 3 ? launch_hp_prolong_add3<T>(k, L.n_int, d0, u, s) : launch_hp_prolong_add<T>(k, L.n_int, d0, u, s);
}

// z = MG_hp(r, 0) (Algorithm 2); r, z FP64 of size n_dof
template <class T>
void mg_hp_impl(hdg_ctx *ctx, const T *r, T *z, cudaStream_t s) {
    const int J = ctx->n_levels - 1;
    DevLevel &LJ = ctx->L[J];
    const int k = ctx->prm.k;
    if (k == 0) {
        // Algorithm 2 with k = 0 is MG_h on the finest level
        CK(cudaMemcpyAsync(Prec<T>::g(LJ), r, sizeof(T) * ctx->n_dof, cudaMemcpyDeviceToDevice, s));
        mg_h<T>(ctx, J, ctx->prm.m_h, true, s);
        CK(cudaMemcpyAsync(z, Prec<T>::u(LJ), sizeof(T) * ctx->n_dof, cudaMemcpyDeviceToDevice, s));
        return;
    }
    const DevOperator &op = ctx->opk;
    T *res = std::is_same<T, double>::value ? (T *)ctx->kr.p : (T *)ctx->krf.p;
    CK(launch_fill<T>(z, T(0), ctx->n_dof, s));
    if (ctx->prm.hp_additive) {
        // additive form (Remark 3.4): the symmetric relaxation of r plus the lowest-order
        // correction of r itself
        for (int j = 0; j < ctx->prm.m_p; ++j) sweep<T>(ctx, LJ, op, r, z, false, s);
        for (int j = 0; j < ctx->prm.m_p; ++j) sweep<T>(ctx, LJ, op, r, z, true, s);
        CK(hp_restrict_any<T>(LJ, k, r, Prec<T>::g(LJ), s));
        mg_h<T>(ctx, J, ctx->prm.m_h, true, s);
        CK(hp_prolong_any<T>(LJ, k, Prec<T>::u(LJ), z, s));
        return;
    }
    for (int j = 0; j < ctx->prm.m_p; ++j) sweep<T>(ctx, LJ, op, r, z, false, s);
    apply_op<T>(ctx, LJ, op, z, r, res, s);
    CK(hp_restrict_any<T>(LJ, k, res, Prec<T>::g(LJ), s));
    mg_h<T>(ctx, J, ctx->prm.m_h, true, s);
    CK(hp_prolong_any<T>(LJ, k, Prec<T>::u(LJ), z, s));
    for (int j = 0; j < ctx->prm.m_p; ++j) sweep<T>(ctx, LJ, op, r, z, true, s);
}

void precond_direct(hdg_ctx *ctx, const double *r, double *z, cudaStream_t s) {
    if (ctx->prm.precision == HDG_FP64) {
        mg_hp_impl<double>(ctx, r, z, s);
    } else {
        CK(launch_d2f(r, ctx->kgf.p, ctx->n_dof, s));
        mg_hp_impl<float>(ctx, ctx->kgf.p, ctx->kuf.p, s);
        CK(launch_f2d(ctx->kuf.p, z, ctx->n_dof, s));
    }
}

void drop_graph(hdg_ctx *ctx) {
    if (ctx->pc_exec) cudaGraphExecDestroy(ctx->pc_exec);
    ctx->pc_exec = nullptr;
    ctx->pc_prec = -1;
    ctx->pc_kernels = 0;
    if (ctx->pcm_exec) cudaGraphExecDestroy(ctx->pcm_exec);
    ctx->pcm_exec = nullptr;
    ctx->pcm_prec = -1;
    ctx->pcm_R = 0;
    ctx->pcm_kernels = 0;
}

// z = MG_hp(r): replays a CUDA graph of the whole preconditioner (several hundred
// small launches per application on deep hierarchies) captured once per
// condensation, with fixed staging buffers; direct launches when the caller's
// stream is itself being captured.
void precond(hdg_ctx *ctx, const double *r, double *z, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone) {
        precond_direct(ctx, r, z, s);
        return;
    }
    const size_t bytes = sizeof(double) * ctx->n_dof;
    if (!ctx->pc_exec || ctx->pc_prec != (int)ctx->prm.precision) {
        drop_graph(ctx);
        dalloc(ctx, ctx->pc_in, ctx->n_dof);
        dalloc(ctx, ctx->pc_out, ctx->n_dof);
        if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
        // the capture stream starts after everything already queued on s
        cudaEvent_t ev;
        CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        CK(cudaEventRecord(ev, s));
        CK(cudaStreamWaitEvent(ctx->cap_stream, ev, 0));
        CK(cudaEventDestroy(ev));
        cudaStream_t cs2 = ctx->cap_stream;
        const unsigned long long l0 = thread_launch_count();
        CK(cudaStreamBeginCapture(cs2, cudaStreamCaptureModeThreadLocal));
        cudaGraph_t g = nullptr;
        try {
            precond_direct(ctx, ctx->pc_in.p, ctx->pc_out.p, cs2);
        } catch (...) {
            cudaStreamEndCapture(cs2, &g);
            if (g) cudaGraphDestroy(g);
            throw;
        }
        CK(cudaStreamEndCapture(cs2, &g));
        cudaError_t e = cudaGraphInstantiate(&ctx->pc_exec, g, 0);
        cudaGraphDestroy(g);
        CK(e);
        ctx->pc_kernels = (long long)(thread_launch_count() - l0);
        note_launches(-ctx->pc_kernels);          // captured, not executed
        ctx->pc_prec = (int)ctx->prm.precision;
    }
    CK(cudaMemcpyAsync(ctx->pc_in.p, r, bytes, cudaMemcpyDeviceToDevice, s));
    CK(cudaGraphLaunch(ctx->pc_exec, s));
    note_launches(ctx->pc_kernels);
    CK(cudaMemcpyAsync(z, ctx->pc_out.p, bytes, cudaMemcpyDeviceToDevice, s));
}

void apply_k(hdg_ctx *ctx, const double *x, const double *g, double *y, cudaStream_t s) {
    DevLevel &LJ = ctx->L[ctx->n_levels - 1];
    CK(launch_apply<double>(LJ, ctx->opk, ctx->opk.A.p, x, g, y, s));
}

double norm2(hdg_ctx *ctx, const double *x, int64_t n, cudaStream_t s) {
    SmallLayout Ly{ctx->restart_alloc};
    CK(launch_dots(x, 1, 0, x, n, ctx->partials.p, s));
    CK(launch_reduce_partials(ctx->partials.p, 1, ctx->small.p + Ly.nrm2(), 0, s));
    return std::sqrt(std::max(read_scalar(ctx, ctx->small.p + Ly.nrm2(), s), 0.0));
}

void ensure_krylov(hdg_ctx *ctx, int R) {
    const int64_t n = ctx->n_dof;
    if (ctx->restart_alloc != R || ctx->V.n < (size_t)(R + 1) * n) {
        dfree(ctx->V);
        dfree(ctx->Z);
        dfree(ctx->small);
        dalloc(ctx, ctx->V, (size_t)(R + 1) * n);
        dalloc(ctx, ctx->Z, (size_t)R * n);
        SmallLayout Ly{R};
        dalloc(ctx, ctx->small, (size_t)Ly.total());
        ctx->restart_alloc = R;
    }
    dalloc(ctx, ctx->w, n);
    dalloc(ctx, ctx->partials, (size_t)(MAX_RESTART + 2) * krylov_partial_blocks());
}

struct FgmresOut {
    int its;
    double res;
    bool stagnated;
};

// flexible GMRES on A^eps x = b: stop at |r| <= max(rtol |r0|, atol).  A restart cycle that
// ended because the Givens estimate reached the tolerance while the true residual did not
// is the mark of round-off in the residual (Remark 3.1: the augmented-Lagrangian term
// magnifies it); when the next such cycle reduces the true residual by less than half, the
// solve stops as stagnated at the attainable level.
FgmresOut fgmres(hdg_ctx *ctx, const double *b, double *x, double rtol, double atol, int R,
                 int max_it, cudaStream_t s) {
    const int64_t n = ctx->n_dof;
    SmallLayout Ly{R};
    double *V = ctx->V.p, *Z = ctx->Z.p, *w = ctx->w.p, *sm = ctx->small.p, *pt = ctx->partials.p;
    int total = 0;
    double tol = -1.0, beta = 0.0, beta_prev = -1.0;
    bool est_reached = false, stagnated = false;
    while (true) {
        apply_k(ctx, x, b, V, s);   // V0 = b - A x
        CK(launch_dots(V, 1, 0, V, n, pt, s));
        CK(launch_reduce_partials(pt, 1, sm + Ly.nrm2(), 0, s));
        beta = std::sqrt(std::max(read_scalar(ctx, sm + Ly.nrm2(), s), 0.0));
        if (!std::isfinite(beta)) {
            ctx->err = "non-finite residual";
            throw Fail{HDG_ERR_NONFINITE};
        }
        if (tol < 0) tol = std::max(rtol * beta, atol);
        if (beta <= tol || total >= max_it) break;
        if (est_reached && beta_prev >= 0 && beta > 0.5 * beta_prev) {
            stagnated = true;
            break;
        }
        beta_prev = beta;
        est_reached = false;
        CK(launch_init_cycle(V, V, n, sm, R, s));
        int m = 0;
        for (int j = 0; j < R; ++j) {
            double *vj = V + (size_t)j * n, *zj = Z + (size_t)j * n;
            precond(ctx, vj, zj, s);
            apply_k(ctx, zj, nullptr, w, s);
            CK(launch_dots(V, j + 1, n, w, n, pt, s));
            CK(launch_reduce_partials(pt, j + 1, sm + Ly.h1(), 0, s));
            CK(launch_update_dots(V, j + 1, n, w, n, sm + Ly.h1(), pt, 1, s));
            CK(launch_reduce_partials(pt, j + 1, sm + Ly.h2(), 0, s));
            CK(launch_update_dots(V, j + 1, n, w, n, sm + Ly.h2(), pt, 2, s));
            CK(launch_reduce_partials(pt, 1, sm + Ly.nrm2(), 0, s));
            CK(launch_givens(sm, j, R, nullptr, s));
            CK(launch_scale_next(w, V + (size_t)(j + 1) * n, n, sm, j, R, s));
            CK(cudaMemcpyAsync(ctx->h_pinned, sm + Ly.res(), 2 * sizeof(double),
                               cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            double res = ctx->h_pinned[0], hn = ctx->h_pinned[1];
            ++total;
            m = j + 1;
            if (!std::isfinite(res)) {
                ctx->err = "non-finite residual estimate";
                throw Fail{HDG_ERR_NONFINITE};
            }
            if (res <= tol) est_reached = true;
            if (res <= tol || total >= max_it || hn == 0.0) break;
        }
        CK(launch_solve_update(sm, m, R, Z, n, x, n, s));
    }
    return {total, beta, stagnated};
}

// preconditioned conjugate gradients on A^eps x = b (Section 5, the paper's Krylov method for
// the generalized Stokes problem; symmetric operator and preconditioner): stop when the
// recursively updated residual has |r| <= max(rtol |r0|, atol).  Work vectors r, z, p, q
// lie consecutively in pcg_buf, so one dot pass gives r.r and z.r together.
FgmresOut pcg(hdg_ctx *ctx, const double *b, double *x, double rtol, double atol, int max_it, cudaStream_t s) {
    const int64_t n = ctx->n_dof;
    dalloc(ctx, ctx->pcg_buf, (size_t)4 * std::max<int64_t>(n, 1));
    double *r = ctx->pcg_buf.p, *z = r + n, *p = z + n, *q = p + n;
    SmallLayout Ly{ctx->restart_alloc};
    double *pt = ctx->partials.p, *sc = ctx->small.p + Ly.h1();
    auto dots2 = [&](const double *w, int nv, double *out) {   // out[j] = (r + j n) . w
        CK(launch_dots(r, nv, n, w, n, pt, s));
        CK(launch_reduce_partials(pt, nv, sc, 0, s));
        CK(cudaMemcpyAsync(ctx->h_pinned, sc, nv * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        for (int j = 0; j < nv; ++j) out[j] = ctx->h_pinned[j];
    };
    apply_k(ctx, x, b, r, s);   // r = b - A x
    double v[2];
    dots2(r, 1, v);
    double rn = std::sqrt(std::max(v[0], 0.0));
    if (!std::isfinite(rn)) {
        ctx->err = "non-finite residual";
        throw Fail{HDG_ERR_NONFINITE};
    }
    const double tol = std::max(rtol * rn, atol);
    if (rn <= tol) return {0, rn, false};
    precond(ctx, r, z, s);
    CK(cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    dots2(z, 1, v);
    double rz = v[0];
    int its = 0;
    while (its < max_it) {
        apply_k(ctx, p, nullptr, q, s);
        CK(launch_dots(p, 1, 0, q, n, pt, s));
        CK(launch_reduce_partials(pt, 1, sc, 0, s));
        const double pq = read_scalar(ctx, sc, s);
        if (!(pq > 0) || !std::isfinite(pq)) {
            ctx->err = "PCG: the operator or the preconditioner is not positive definite (p.Ap = " +
                       std::to_string(pq) + ")";
            throw Fail{HDG_ERR_BREAKDOWN};
        }
        const double alpha = rz / pq;
        CK(launch_axpby(alpha, p, 1.0, x, n, s));
        CK(launch_axpby(-alpha, q, 1.0, r, n, s));
        ++its;
        dots2(r, 1, v);
        rn = std::sqrt(std::max(v[0], 0.0));
        if (!std::isfinite(rn)) {
            ctx->err = "non-finite residual";
            throw Fail{HDG_ERR_NONFINITE};
        }
        if (rn <= tol) break;
        precond(ctx, r, z, s);
        dots2(r, 2, v);   // v[1] = z . r
        const double beta = v[1] / rz;
        rz = v[1];
        CK(launch_axpby(1.0, z, beta, p, n, s));
    }
    return {its, rn, false};
}

const double *cell_nu_of(hdg_ctx *ctx, int l) {
    return ctx->prm.nu_elem ? ctx->L[l].cell_nu.p : nullptr;
}

// finest-level convecting field (library copy), NULL for the generalized Stokes problem
const double *conv_of(hdg_ctx *ctx) { return ctx->has_conv ? ctx->conv_k.p : nullptr; }

// previous skeleton iterate of a Newton step (library copy), or NULL
const double *newton_of(hdg_ctx *ctx) { return ctx->has_newton ? ctx->newton_x.p : nullptr; }

// condensed load F from lattice forcing (the element matrices are left untouched)
void load_impl(hdg_ctx *ctx, const double *forcing, double *rhs_out, cudaStream_t s) {
    DevLevel &LJ = ctx->L[ctx->n_levels - 1];
    if (ctx->dim == 3) {
        int sms = 0;
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
        const int blocks = 2 * std::max(sms, 1);   // the condensation's workspace (sized for this k)
        CK(launch_condense3(ctx->prm.k, LJ, ctx->ref3k_dev.p, ctx->ref3k, ctx->prm.nu, nullptr, ctx->prm.beta,
                            ctx->prm.gamma, forcing, nullptr, nullptr, ctx->opk.Fel.p, ctx->c3_scratch.p, blocks,
                            ctx->status_flag.p, s));
        CK(launch_assemble_load(LJ, ctx->opk, rhs_out, s));
        if (ctx->has_dir) CK(launch_dirichlet_load(LJ, ctx->opk, ctx->dir_x.p, rhs_out, s));
        return;
    }
    CK(launch_condense(ctx->prm.k, LJ, ctx->refk_dev.p, ctx->refk, ctx->prm.nu, cell_nu_of(ctx, ctx->n_levels - 1),
                       ctx->prm.beta, ctx->prm.gamma, forcing, conv_of(ctx), ctx->conv_t, newton_of(ctx), nullptr,
                       nullptr, ctx->opk.Fel.p, ctx->status_flag.p, RecoverArgs(), s));
    CK(launch_assemble_load(LJ, ctx->opk, rhs_out, s));
    if (ctx->has_dir) CK(launch_dirichlet_load(LJ, ctx->opk, ctx->dir_x.p, rhs_out, s));
}

void recover_impl(hdg_ctx *ctx, const double *u, const double *forcing, double *L, double *rt, double *ulat,
                  cudaStream_t s) {
    DevLevel &LJ = ctx->L[ctx->n_levels - 1];
    RecoverArgs rec;
    rec.x = u;
    rec.cell_int = LJ.cell_int.p;
    rec.cell_bnd = LJ.cell_bnd.p;
    rec.xD = ctx->has_dir ? ctx->dir_x.p : nullptr;
    rec.L = L;
    rec.rt = rt;
    rec.ulat = ulat;
    CK(launch_condense(ctx->prm.k, LJ, ctx->refk_dev.p, ctx->refk, ctx->prm.nu, cell_nu_of(ctx, ctx->n_levels - 1),
                       ctx->prm.beta, ctx->prm.gamma, forcing, conv_of(ctx), ctx->conv_t, newton_of(ctx), nullptr,
                       nullptr, nullptr, ctx->status_flag.p, rec, s));
}

// Augmented-Lagrangian Uzawa loop with FGMRES inner solves (eq. stOpEq-ALU); returns
// HDG_OK or HDG_ERR_NOT_CONVERGED, throws on other failures
hdg_status uzawa_solve(hdg_ctx *ctx, const double *F, double *u, double *p, const hdg_solve_opts *opts_in,
                       hdg_solve_info &loc, cudaStream_t s) {
    hdg_status conv = HDG_OK;
    hdg_solve_opts o;
    hdg_default_solve_opts(&o);
    if (opts_in) o = *opts_in;
    REQUIRE(o.restart >= 1 && o.restart <= MAX_RESTART, "restart out of range 1..64");
    REQUIRE(o.max_uzawa >= 1 && o.max_uzawa <= 64, "max_uzawa out of range 1..64");
    REQUIRE(o.max_it >= 1 && o.rtol >= 0 && o.atol >= 0 && o.floor_rel >= 0 && o.uzawa_tol >= 0,
            "bad tolerances");
    REQUIRE(o.krylov == 0 || o.krylov == 1, "krylov must be 0 (FGMRES) or 1 (PCG)");
    REQUIRE(o.krylov == 0 || (!ctx->has_conv && (ctx->prm.precision == HDG_FP64 ||
                                                 ctx->prm.precision == HDG_MIXED_FP32)),
            "PCG needs a symmetric operator and preconditioner: no convection, FP64 or FP32 preconditioner");
    ensure_krylov(ctx, o.restart);
    const int J = ctx->n_levels - 1;
    DevLevel &LJ = ctx->L[J];
    const int k = ctx->prm.k;
    const double normF = norm2(ctx, F, ctx->n_dof, s);
    loc = hdg_solve_info{};
    loc.normF = normF;
    // inner floor: floor_rel |F| (and atol), raised to twice the residual at which an inner
    // solve stagnated on round-off, so that later Uzawa steps do not chase it again
    double floor_abs = std::max(o.floor_rel * normF, o.atol);
    double *g = ctx->kt.p;
    double ndp_prev = -1.0;
    bool done = false;
    for (int it = 0; it < o.max_uzawa; ++it) {
        CK(launch_uzawa_rhs(LJ, k, F, p, g, s));
        FgmresOut fo = o.krylov == 1 ? pcg(ctx, g, u, o.rtol, floor_abs, o.max_it, s)
                                     : fgmres(ctx, g, u, o.rtol, floor_abs, o.restart, o.max_it, s);
        loc.krylov_its[it] = fo.its;
        loc.krylov_its_total += fo.its;
        loc.uzawa_its = it + 1;
        loc.res_mom = fo.res;
        if (fo.its >= o.max_it) conv = HDG_ERR_NOT_CONVERGED;
        if (fo.stagnated) floor_abs = std::max(floor_abs, 2.0 * fo.res);
        loc.res_floor = floor_abs;
        CK(launch_uzawa_update(LJ, k, u, p, ctx->prm.gamma, ctx->prm.nu, cell_nu_of(ctx, J),
                               ctx->has_dir ? ctx->dir_flux.p : nullptr, ctx->partials.p, s));
        SmallLayout Ly{o.restart};
        CK(launch_reduce_partials(ctx->partials.p, 4, ctx->small.p + Ly.h1(), 0, s));
        CK(cudaMemcpyAsync(ctx->h_pinned, ctx->small.p + Ly.h1(), 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        const double ndp = std::sqrt(std::max(ctx->h_pinned[0], 0.0));
        const double npn = std::sqrt(std::max(ctx->h_pinned[1], 0.0));
        loc.div_l2 = std::sqrt(std::max(ctx->h_pinned[3], 0.0));
        loc.dp_rel = npn > 0 ? ndp / npn : 0.0;
        if (!std::isfinite(ndp) || !std::isfinite(npn)) {
            ctx->err = "non-finite pressure update";
            throw Fail{HDG_ERR_NONFINITE};
        }
        if (ndp <= o.atol || (it > 0 && fo.its == 0)) { done = true; break; }
        if (ndp_prev >= 0) {
            double rho = std::min(ndp / ndp_prev, 0.99);
            if (rho / (1.0 - rho) * ndp <= o.uzawa_tol * npn) { done = true; break; }
        }
        ndp_prev = ndp;
    }
    if (!done && conv == HDG_OK) conv = HDG_ERR_NOT_CONVERGED;
    return conv;
}

double device_sum(hdg_ctx *ctx, const double *x, int64_t n, cudaStream_t s) {
    SmallLayout Ly{ctx->restart_alloc};
    CK(launch_sum(x, n, ctx->partials.p, s));
    CK(launch_reduce_partials(ctx->partials.p, 1, ctx->small.p + Ly.nrm2(), 0, s));
    return read_scalar(ctx, ctx->small.p + Ly.nrm2(), s);
}

// ===================================================================== multi-RHS
// R columns (a power of two, the caller's nrhs padded with zero columns) run
// the same Algorithms 1 and 2, FGMRES and Uzawa steps as the single solve, in
// lockstep: every kernel works on multi-vectors [rows][R], and each column keeps
// its own Krylov least-squares problem, tolerances and stopping decisions.

int pad_width(int nrhs) {
    int R = 1;
    while (R < nrhs) R <<= 1;
    return R;
}

template <class T>
struct PrecM;
template <>
struct PrecM<double> {
    static double *g(DevLevel &L) { return L.mg.p; }
    static double *u(DevLevel &L) { return L.mu.p; }
    static double *r(DevLevel &L) { return L.mr.p; }
    static double *t(DevLevel &L) { return L.mt.p; }
    static double *c1(DevLevel &L) { return L.mc1.p; }
    static double *c2(DevLevel &L) { return L.mc2.p; }
    static void alloc(hdg_ctx *ctx, DevLevel &L, int R) {
        const size_t n = (size_t)std::max<int64_t>(2 * L.n_int, 1) * R;
        dalloc(ctx, L.mg, n); dalloc(ctx, L.mu, n); dalloc(ctx, L.mr, n); dalloc(ctx, L.mt, n);
        dalloc(ctx, L.mc1, (size_t)std::max<int64_t>(12 * L.nc_coarse, 1) * R);
        dalloc(ctx, L.mc2, (size_t)std::max<int64_t>(6 * L.nc_coarse, 1) * R);
    }
};
template <>
struct PrecM<float> {
    static float *g(DevLevel &L) { return L.mgf.p; }
    static float *u(DevLevel &L) { return L.muf.p; }
    static float *r(DevLevel &L) { return L.mrf.p; }
    static float *t(DevLevel &L) { return L.mtf.p; }
    static float *c1(DevLevel &L) { return L.mc1f.p; }
    static float *c2(DevLevel &L) { return L.mc2f.p; }
    static void alloc(hdg_ctx *ctx, DevLevel &L, int R) {
        const size_t n = (size_t)std::max<int64_t>(2 * L.n_int, 1) * R;
        dalloc(ctx, L.mgf, n); dalloc(ctx, L.muf, n); dalloc(ctx, L.mrf, n); dalloc(ctx, L.mtf, n);
        dalloc(ctx, L.mc1f, (size_t)std::max<int64_t>(12 * L.nc_coarse, 1) * R);
        dalloc(ctx, L.mc2f, (size_t)std::max<int64_t>(6 * L.nc_coarse, 1) * R);
    }
};

// tile of the batched order-k sweep for this precision and width (0, 0 = defaults)
template <class T>
void tile_of(const hdg_ctx *ctx, int R, int &rb, int &nt) {
    if (ctx->tile_force_rb || ctx->tile_force_nt) {
        rb = ctx->tile_force_rb;
        nt = ctx->tile_force_nt;
        return;
    }
    const int pi = std::is_same<T, double>::value ? 0 : 1, li = log2_width(R);
    rb = ctx->tile_rb[pi][li];
    nt = ctx->tile_nt[pi][li];
}

// Autotuner of the batched order-k sweep on CUDA cores: times one colour phase of the
// finest level (the colour with the most patches) on scratch vectors for every rows-
// per-thread / block-size pair and keeps the fastest for this precision and width.
// The pairs give bitwise-identical results (each row's sums run in the same order).
template <class T>
void tune_gs_m(hdg_ctx *ctx, int R, cudaStream_t s) {
    const int pi = std::is_same<T, double>::value ? 0 : 1, li = log2_width(R);
    const DevLevel &L = ctx->L[ctx->n_levels - 1];
    const DevOperator &op = ctx->opk;
    const size_t n = (size_t)std::max<int64_t>(ctx->n_dof, 1) * R;
    dalloc(ctx, ctx->tune_buf, sizeof(T) == sizeof(double) ? 2 * n : n);   // two T vectors of n values
    T *g = reinterpret_cast<T *>(ctx->tune_buf.p), *u = g + n;
    CK(cudaMemsetAsync(ctx->tune_buf.p, 0, 2 * n * sizeof(T), s));
    int colour = 0;
    for (int c = 1; c < L.n_colours; ++c)
        if (L.colour_ptr[c + 1] - L.colour_ptr[c] > L.colour_ptr[colour + 1] - L.colour_ptr[colour]) colour = c;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    double best = 1e300;
    int brb = 0, bnt = 0;
    for (int rb : {1, 2, 4}) {
        if (op.dpf % rb) continue;
        for (int nt : {128, 256}) {
            CK(launch_gs_colour_m<T>(L, op, R, Prec<T>::A(op), Prec<T>::P(op), colour, g, u, s, rb, nt));
            CK(cudaEventRecord(e0, s));
            for (int it = 0; it < 3; ++it)
                CK(launch_gs_colour_m<T>(L, op, R, Prec<T>::A(op), Prec<T>::P(op), colour, g, u, s, rb, nt));
            CK(cudaEventRecord(e1, s));
            CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            if (ms / 3 < best) {
                best = ms / 3;
                brb = rb;
                bnt = nt;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->tile_rb[pi][li] = brb;
    ctx->tile_nt[pi][li] = bnt;
    ctx->tile_ms[pi][li] = best;
}

// Autotuner of the tensor-core sweep: times the largest colour phase of the finest level for
// 128 and 256 threads per block and keeps the faster.  Every tile's MMAs and the column
// maxima are the same for both block sizes, so the results are bitwise identical.
void tune_gs_tc(hdg_ctx *ctx, int R, cudaStream_t s) {
    const int li = log2_width(R);
    const DevLevel &L = ctx->L[ctx->n_levels - 1];
    const DevOperator &op = ctx->opk;
    const size_t n = (size_t)std::max<int64_t>(ctx->n_dof, 1) * R;
    dalloc(ctx, ctx->tune_buf, n);   // two FP32 vectors of n values
    float *g = reinterpret_cast<float *>(ctx->tune_buf.p), *u = g + n;
    CK(cudaMemsetAsync(ctx->tune_buf.p, 0, 2 * n * sizeof(float), s));
    int colour = 0;
    for (int c = 1; c < L.n_colours; ++c)
        if (L.colour_ptr[c + 1] - L.colour_ptr[c] > L.colour_ptr[colour + 1] - L.colour_ptr[colour]) colour = c;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    double best = 1e300;
    int bnt = 256;
    for (int nt : {128, 256}) {
        CK(launch_gs_colour_tc(L, op, R, colour, g, u, s, nt));
        CK(cudaEventRecord(e0, s));
        for (int it = 0; it < 3; ++it) CK(launch_gs_colour_tc(L, op, R, colour, g, u, s, nt));
        CK(cudaEventRecord(e1, s));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (ms / 3 < best) {
            best = ms / 3;
            bnt = nt;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->tile_tc_nt[li] = bnt;
    ctx->tile_tc_ms[li] = best;
}

// tunes the batched order-k sweep (CUDA-core tile, or the tensor-core block size) of the
// current precision for width R unless it is done or forced; false if the stream is capturing
bool ensure_tuned(hdg_ctx *ctx, int R, cudaStream_t s) {
    if (ctx->tile_force_rb || ctx->tile_force_nt || ctx->prm.k == 0) return true;
    const bool fp64 = ctx->prm.precision == HDG_FP64;
    const bool tc = !fp64 && gs_tc_supported(ctx->L[ctx->n_levels - 1], ctx->opk, R);
    if (tc ? ctx->tile_tc_nt[log2_width(R)] != 0 : ctx->tile_rb[fp64 ? 0 : 1][log2_width(R)] != 0) return true;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone) return false;
    if (tc) tune_gs_tc(ctx, R, s);
    else if (fp64) tune_gs_m<double>(ctx, R, s);
    else tune_gs_m<float>(ctx, R, s);
    return true;
}

// the batched forms run Algorithm 2 with block GS only
void require_multi_variant(hdg_ctx *ctx) {
    if (ctx->prm.smoother != 0 || ctx->prm.hp_additive) {
        ctx->err = "batched (_multi) calls support the block GS smoother and Algorithm 2 only";
        throw Fail{HDG_ERR_UNSUPPORTED};
    }
}

template <class T>
void sweep_m(hdg_ctx *ctx, const DevLevel &L, const DevOperator &op, int R, const T *g, T *u, bool reverse,
             cudaStream_t s) {
    require_multi_variant(ctx);
    int rb = 0, nt = 0;
    if (&op == &ctx->opk) tile_of<T>(ctx, R, rb, nt);
    bool tc = false;
    if constexpr (std::is_same<T, float>::value) tc = gs_tc_supported(L, op, R);
    for (int i = 0; i < L.n_colours; ++i) {
        const int c = reverse ? L.n_colours - 1 - i : i;
        if constexpr (std::is_same<T, float>::value) {
            if (tc) {
                const int tnt = ctx->tile_force_nt ? ctx->tile_force_nt : ctx->tile_tc_nt[log2_width(R)];
                CK(launch_gs_colour_tc(L, op, R, c, g, u, s, tnt));
                continue;
            }
        }
        CK(launch_gs_colour_m<T>(L, op, R, Prec<T>::A(op), Prec<T>::P(op), c, g, u, s, rb, nt));
    }
}

template <class T>
void mg_h_m(hdg_ctx *ctx, int l, int m, bool zero_init, int R, cudaStream_t s) {
    DevLevel &L = ctx->L[l];
    if (l == 0) {
        CK(launch_coarse_apply_m<T>(ctx->coarse_inv.p, 2 * L.n_int, R, PrecM<T>::g(L), PrecM<T>::u(L), s));
        return;
    }
    DevLevel &C = ctx->L[l - 1];
    const int64_t n = 2 * L.n_int * R;
    T *g = PrecM<T>::g(L), *u = PrecM<T>::u(L), *r = PrecM<T>::r(L);
    if (zero_init) CK(cudaMemsetAsync(u, 0, sizeof(T) * n, s));
    for (int j = 0; j < m; ++j) sweep_m<T>(ctx, L, L.op0, R, g, u, false, s);
    CK(launch_apply_m<T>(L, L.op0, R, Prec<T>::A(L.op0), u, g, r, s));
    CK(launch_restrict_m<T>(L, C, R, Prec<T>::W(L), Prec<T>::H(L), r, PrecM<T>::c1(L), PrecM<T>::c2(L),
                            PrecM<T>::g(C), s));
    const int q = ctx->prm.cycle;
    const int mc = (q == 1) ? m * ctx->prm.vcycle_growth : m;
    for (int it = 0; it < q; ++it) mg_h_m<T>(ctx, l - 1, mc, it == 0, R, s);
    CK(launch_prolong_add_m<T>(L, C, R, Prec<T>::W(L), Prec<T>::H(L), PrecM<T>::u(C), PrecM<T>::t(L), u, s));
    for (int j = 0; j < m; ++j) sweep_m<T>(ctx, L, L.op0, R, g, u, true, s);
}

// z = MG_hp(r, 0) for R columns (r, z of type T, [n_dof][R])
template <class T>
void mg_hp_m(hdg_ctx *ctx, const T *r, T *z, T *res, int R, cudaStream_t s) {
    const int J = ctx->n_levels - 1;
    DevLevel &LJ = ctx->L[J];
    const int k = ctx->prm.k;
    const size_t bytes = sizeof(T) * ctx->n_dof * R;
    if (k == 0) {
        CK(cudaMemcpyAsync(PrecM<T>::g(LJ), r, bytes, cudaMemcpyDeviceToDevice, s));
        mg_h_m<T>(ctx, J, ctx->prm.m_h, true, R, s);
        CK(cudaMemcpyAsync(z, PrecM<T>::u(LJ), bytes, cudaMemcpyDeviceToDevice, s));
        return;
    }
    const DevOperator &op = ctx->opk;
    CK(cudaMemsetAsync(z, 0, bytes, s));
    for (int j = 0; j < ctx->prm.m_p; ++j) sweep_m<T>(ctx, LJ, op, R, r, z, false, s);
    CK(launch_apply_m<T>(LJ, op, R, Prec<T>::A(op), z, r, res, s));
    CK(launch_hp_restrict_m<T>(k, LJ.n_int, R, res, PrecM<T>::g(LJ), s));
    mg_h_m<T>(ctx, J, ctx->prm.m_h, true, R, s);
    CK(launch_hp_prolong_add_m<T>(k, LJ.n_int, R, PrecM<T>::u(LJ), z, s));
    for (int j = 0; j < ctx->prm.m_p; ++j) sweep_m<T>(ctx, LJ, op, R, r, z, true, s);
}

// work buffers of the multi preconditioner and operator for width R
void ensure_multi_work(hdg_ctx *ctx, int R) {
    const size_t n = (size_t)std::max<int64_t>(ctx->n_dof, 1) * R;
    const bool fp64 = ctx->prm.precision == HDG_FP64;
    for (auto &L : ctx->L) {
        if (fp64) PrecM<double>::alloc(ctx, L, R);
        else PrecM<float>::alloc(ctx, L, R);
    }
    for (const DevLevel *L : {&ctx->L[ctx->n_levels - 1]}) {
        const DevOperator &op = ctx->prm.k > 0 ? ctx->opk : L->op0;
        REQUIRE(gs_m_smem(*L, op, R, fp64 ? 8 : 4) <= 200 * 1024,
                "too many right-hand sides for the patch size (shared memory)");
        REQUIRE(L->nc * (int64_t)op.nloc * op.nloc < ((int64_t)1 << 31), "mesh too large for the batched smoother");
    }
    dalloc(ctx, ctx->mkr, n);
    if (!fp64) {
        dalloc(ctx, ctx->mkgf, n);
        dalloc(ctx, ctx->mkuf, n);
        dalloc(ctx, ctx->mkrf, n);
    }
}

void precond_m_direct(hdg_ctx *ctx, const double *r, double *z, int R, cudaStream_t s) {
    const int64_t n = ctx->n_dof * R;
    if (ctx->prm.precision == HDG_FP64) {
        mg_hp_m<double>(ctx, r, z, ctx->mkr.p, R, s);
    } else {
        CK((launch_convert_m<double, float>(r, ctx->mkgf.p, n, s)));
        mg_hp_m<float>(ctx, ctx->mkgf.p, ctx->mkuf.p, ctx->mkrf.p, R, s);
        CK((launch_convert_m<float, double>(ctx->mkuf.p, z, n, s)));
    }
}

// z = MG_hp(r) for R columns through a CUDA graph captured once per (precision, R)
void precond_m(hdg_ctx *ctx, const double *r, double *z, int R, cudaStream_t s) {
    require_multi_variant(ctx);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(s, &cs));
    ensure_multi_work(ctx, R);
    ensure_tuned(ctx, R, s);
    if (cs != cudaStreamCaptureStatusNone) {
        precond_m_direct(ctx, r, z, R, s);
        return;
    }
    const size_t bytes = sizeof(double) * ctx->n_dof * R;
    if (!ctx->pcm_exec || ctx->pcm_prec != (int)ctx->prm.precision || ctx->pcm_R != R) {
        if (ctx->pcm_exec) cudaGraphExecDestroy(ctx->pcm_exec);
        ctx->pcm_exec = nullptr;
        dalloc(ctx, ctx->pcm_in, ctx->n_dof * R);
        dalloc(ctx, ctx->pcm_out, ctx->n_dof * R);
        if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
        cudaEvent_t ev;
        CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        CK(cudaEventRecord(ev, s));
        CK(cudaStreamWaitEvent(ctx->cap_stream, ev, 0));
        CK(cudaEventDestroy(ev));
        cudaStream_t cs2 = ctx->cap_stream;
        const unsigned long long l0 = thread_launch_count();
        CK(cudaStreamBeginCapture(cs2, cudaStreamCaptureModeThreadLocal));
        cudaGraph_t g = nullptr;
        try {
            precond_m_direct(ctx, ctx->pcm_in.p, ctx->pcm_out.p, R, cs2);
        } catch (...) {
            cudaStreamEndCapture(cs2, &g);
            if (g) cudaGraphDestroy(g);
            throw;
        }
        CK(cudaStreamEndCapture(cs2, &g));
        cudaError_t e = cudaGraphInstantiate(&ctx->pcm_exec, g, 0);
        cudaGraphDestroy(g);
        CK(e);
        ctx->pcm_kernels = (long long)(thread_launch_count() - l0);
        note_launches(-ctx->pcm_kernels);
        ctx->pcm_prec = (int)ctx->prm.precision;
        ctx->pcm_R = R;
    }
    CK(cudaMemcpyAsync(ctx->pcm_in.p, r, bytes, cudaMemcpyDeviceToDevice, s));
    CK(cudaGraphLaunch(ctx->pcm_exec, s));
    note_launches(ctx->pcm_kernels);
    CK(cudaMemcpyAsync(z, ctx->pcm_out.p, bytes, cudaMemcpyDeviceToDevice, s));
}

void ensure_krylov_m(hdg_ctx *ctx, int Rst, int R) {
    const size_t n = (size_t)std::max<int64_t>(ctx->n_dof, 1) * R;
    SmallLayout Ly{Rst};
    if (ctx->mRst != Rst || ctx->mR != R || ctx->mV.n < (size_t)(Rst + 1) * n) {
        dfree(ctx->mV);
        dfree(ctx->mZ);
        dalloc(ctx, ctx->mV, (size_t)(Rst + 1) * n);
        dalloc(ctx, ctx->mZ, (size_t)Rst * n);
        ctx->mRst = Rst;
        ctx->mR = R;
    }
    dalloc(ctx, ctx->msmall, (size_t)Ly.total() * R);
    dalloc(ctx, ctx->mhbuf, (size_t)(Rst + 2) * R);
    dalloc(ctx, ctx->mw, n);
    dalloc(ctx, ctx->mG, n);
    dalloc(ctx, ctx->mpart, (size_t)(MAX_RESTART + 2) * R * krylov_m_blocks());
    dalloc(ctx, ctx->mint, 2 * (size_t)R);
    if (!ctx->h_multi) CK(cudaMallocHost((void **)&ctx->h_multi, sizeof(double) * 4 * MAX_NRHS));
}

// per-column squared norms of x ([n][R]) -> host out[r]
void norms2_m(hdg_ctx *ctx, const double *x, int64_t n, int R, double *out, cudaStream_t s) {
    SmallLayout Ly{ctx->mRst};
    const int stride = Ly.total();
    CK(launch_dots_m(x, 1, 0, x, n * R, R, ctx->mpart.p, s));
    CK(launch_reduce_partials_m(ctx->mpart.p, 1, R, ctx->msmall.p, stride, Ly.nrm2(), nullptr, s));
    CK(cudaMemcpy2DAsync(ctx->h_multi, sizeof(double), ctx->msmall.p + Ly.nrm2(), sizeof(double) * stride,
                         sizeof(double), R, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int r = 0; r < R; ++r) out[r] = ctx->h_multi[r];
}

struct FgmresOutM {
    int its;                    // lockstep iterations
    std::vector<int> its_r;     // iterations each column was active
    std::vector<double> res_r;  // last true residual norm per column
    std::vector<char> stag_r;   // column stopped as stagnated on round-off (see fgmres)
};

// flexible GMRES on A^eps X = B for R columns; column r stops at |r_r| <= max(rtol |r_r0|, atol_r[r])
FgmresOutM fgmres_m(hdg_ctx *ctx, const double *b, double *x, double rtol, const std::vector<double> &atol_r,
                    const std::vector<char> &skip, int Rst, int max_it, int R, cudaStream_t s) {
    const int64_t n = ctx->n_dof * R;
    SmallLayout Ly{Rst};
    const int stride = Ly.total();
    DevLevel &LJ = ctx->L[ctx->n_levels - 1];
    double *V = ctx->mV.p, *Z = ctx->mZ.p, *w = ctx->mw.p, *sm = ctx->msmall.p, *pt = ctx->mpart.p;
    double *hb = ctx->mhbuf.p;
    FgmresOutM out{0, std::vector<int>(R, 0), std::vector<double>(R, 0.0), std::vector<char>(R, 0)};
    std::vector<double> tol(R, -1.0), beta(R), beta_prev(R, -1.0);
    std::vector<char> est(R, 0);   // the column's last cycle ended on the Givens estimate
    std::vector<int> m_r(R);
    std::vector<char> done(R);
    // outer operator: FP64, or double-FP32 with the mixed preconditioner
    const bool df = ctx->prm.precision != HDG_FP64;
    if (df && !ctx->opk.alo_valid) {
        const size_t na = (size_t)ctx->opk.nloc * ctx->opk.nloc * LJ.nc;
        dalloc(ctx, ctx->opk.Alo, na);
        CK(launch_split_lo(ctx->opk.A.p, ctx->opk.Af.p, ctx->opk.Alo.p, (int64_t)na, s));
        ctx->opk.alo_valid = true;
    }
    if (df) dalloc(ctx, ctx->mxs, (size_t)std::max<int64_t>(n, 1));
    auto outer = [&](const double *xx, const double *gg, double *yy) {
        if (df) CK(launch_apply_df_m(LJ, ctx->opk, R, ctx->opk.Af.p, ctx->opk.Alo.p, xx, ctx->mxs.p, gg, yy, s));
        else CK(launch_apply_m<double>(LJ, ctx->opk, R, ctx->opk.A.p, xx, gg, yy, s));
    };
    while (true) {
        outer(x, b, V);   // V0 = b - A x
        norms2_m(ctx, V, ctx->n_dof, R, beta.data(), s);
        bool any = false;
        for (int r = 0; r < R; ++r) {
            beta[r] = std::sqrt(std::max(beta[r], 0.0));
            if (!std::isfinite(beta[r])) {
                ctx->err = "non-finite residual";
                throw Fail{HDG_ERR_NONFINITE};
            }
            if (tol[r] < 0) tol[r] = std::max(rtol * beta[r], atol_r[r]);
            out.res_r[r] = beta[r];
            done[r] = skip[r] || beta[r] <= tol[r] || out.stag_r[r];
            if (!done[r] && est[r] && beta_prev[r] >= 0 && beta[r] > 0.5 * beta_prev[r]) {
                out.stag_r[r] = 1;
                done[r] = 1;
            }
            if (!done[r]) beta_prev[r] = beta[r];
            est[r] = 0;
            any = any || !done[r];
        }
        if (!any || out.its >= max_it) break;
        CK(launch_init_cycle_m(V, V, n, R, sm, stride, Rst, s));
        std::fill(m_r.begin(), m_r.end(), 0);
        int mmax = 0;
        for (int j = 0; j < Rst; ++j) {
            double *vj = V + (size_t)j * n, *zj = Z + (size_t)j * n;
            precond_m(ctx, vj, zj, R, s);
            outer(zj, nullptr, w);
            CK(launch_dots_m(V, j + 1, n, w, n, R, pt, s));
            CK(launch_reduce_partials_m(pt, j + 1, R, sm, stride, Ly.h1(), hb, s));
            CK(launch_update_dots_m(V, j + 1, n, w, n, R, hb, pt, 1, s));
            CK(launch_reduce_partials_m(pt, j + 1, R, sm, stride, Ly.h2(), hb, s));
            CK(launch_update_dots_m(V, j + 1, n, w, n, R, hb, pt, 2, s));
            CK(launch_reduce_partials_m(pt, 1, R, sm, stride, Ly.nrm2(), nullptr, s));
            CK(launch_givens_m(sm, stride, j, Rst, R, s));
            CK(launch_scale_next_m(w, V + (size_t)(j + 1) * n, n, R, sm, stride, Ly.hn(), s));
            CK(cudaMemcpy2DAsync(ctx->h_multi, 2 * sizeof(double), sm + Ly.res(), sizeof(double) * stride,
                                 2 * sizeof(double), R, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            ++out.its;
            mmax = j + 1;
            bool all = true;
            for (int r = 0; r < R; ++r) {
                if (done[r]) continue;
                const double res = ctx->h_multi[2 * r], hn = ctx->h_multi[2 * r + 1];
                if (!std::isfinite(res)) {
                    ctx->err = "non-finite residual estimate";
                    throw Fail{HDG_ERR_NONFINITE};
                }
                m_r[r] = j + 1;
                out.its_r[r] += 1;
                if (res <= tol[r]) est[r] = 1;
                if (res <= tol[r] || hn == 0.0) done[r] = 1;
                else all = false;
            }
            if (all || out.its >= max_it) break;
        }
        // pageable source: staged before cudaMemcpyAsync returns
        CK(cudaMemcpyAsync(ctx->mint.p, m_r.data(), sizeof(int) * R, cudaMemcpyHostToDevice, s));
        CK(launch_solve_update_m(sm, stride, ctx->mint.p, mmax, Rst, Z, n, x, n, R, s));
    }
    return out;
}

// Uzawa for R columns (eq. stOpEq-ALU), each with the stopping rule of uzawa_solve
hdg_status uzawa_solve_m(hdg_ctx *ctx, int nrhs, int R, const double *F, double *u, double *p,
                         const hdg_solve_opts *opts_in, std::vector<hdg_solve_info> &info, cudaStream_t s) {
    hdg_status conv = HDG_OK;
    hdg_solve_opts o;
    hdg_default_solve_opts(&o);
    if (opts_in) o = *opts_in;
    REQUIRE(o.restart >= 1 && o.restart <= 32, "restart out of range 1..32");
    REQUIRE(o.max_uzawa >= 1 && o.max_uzawa <= 64, "max_uzawa out of range 1..64");
    if (o.krylov != 0) {
        ctx->err = "batched solves run flexible GMRES only (krylov = 0)";
        throw Fail{HDG_ERR_UNSUPPORTED};
    }
    if (ctx->has_dir) {
        ctx->err = "batched solves take homogeneous Dirichlet data only";
        throw Fail{HDG_ERR_UNSUPPORTED};
    }
    REQUIRE(o.max_it >= 1 && o.rtol >= 0 && o.atol >= 0 && o.floor_rel >= 0 && o.uzawa_tol >= 0,
            "bad tolerances");
    ensure_krylov_m(ctx, o.restart, R);
    ensure_multi_work(ctx, R);
    const int J = ctx->n_levels - 1;
    DevLevel &LJ = ctx->L[J];
    const int k = ctx->prm.k;
    std::vector<double> normF(R);
    norms2_m(ctx, F, ctx->n_dof, R, normF.data(), s);
    info.assign(R, hdg_solve_info{});
    std::vector<double> floor_abs(R), ndp_prev(R, -1.0);
    std::vector<char> fin(R, 0);
    for (int r = 0; r < R; ++r) {
        normF[r] = std::sqrt(std::max(normF[r], 0.0));
        info[r].normF = normF[r];
        floor_abs[r] = std::max(o.floor_rel * normF[r], o.atol);
        if (r >= nrhs) fin[r] = 1;
    }
    double *g = ctx->mG.p;
    SmallLayout Ly{o.restart};
    const int stride = Ly.total();
    for (int it = 0; it < o.max_uzawa; ++it) {
        CK(launch_uzawa_rhs_m(LJ, k, R, F, p, g, s));
        FgmresOutM fo = fgmres_m(ctx, g, u, o.rtol, floor_abs, fin, o.restart, o.max_it, R, s);
        std::vector<int> frozen(R);
        for (int r = 0; r < R; ++r) frozen[r] = fin[r];
        CK(cudaMemcpyAsync(ctx->mint.p + R, frozen.data(), sizeof(int) * R, cudaMemcpyHostToDevice, s));
        CK(launch_uzawa_update_m(LJ, k, R, u, p, ctx->prm.gamma, ctx->prm.nu, cell_nu_of(ctx, J), ctx->mint.p + R,
                                 ctx->mpart.p, s));
        CK(launch_reduce_partials_m(ctx->mpart.p, 3, R, ctx->msmall.p, stride, Ly.h1(), nullptr, s));
        CK(cudaMemcpy2DAsync(ctx->h_multi, 3 * sizeof(double), ctx->msmall.p + Ly.h1(), sizeof(double) * stride,
                             3 * sizeof(double), R, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        bool all = true;
        for (int r = 0; r < R; ++r) {
            if (fin[r]) continue;
            hdg_solve_info &in = info[r];
            const int its = fo.its_r[r];
            in.krylov_its[it] = its;
            in.krylov_its_total += its;
            in.uzawa_its = it + 1;
            in.res_mom = fo.res_r[r];
            if (its >= o.max_it) conv = HDG_ERR_NOT_CONVERGED;
            if (fo.stag_r[r]) floor_abs[r] = std::max(floor_abs[r], 2.0 * fo.res_r[r]);
            in.res_floor = floor_abs[r];
            in.div_l2 = -1.0;   // not computed by the batched update
            const double ndp = std::sqrt(std::max(ctx->h_multi[3 * r], 0.0));
            const double npn = std::sqrt(std::max(ctx->h_multi[3 * r + 1], 0.0));
            in.dp_rel = npn > 0 ? ndp / npn : 0.0;
            if (!std::isfinite(ndp) || !std::isfinite(npn)) {
                ctx->err = "non-finite pressure update";
                throw Fail{HDG_ERR_NONFINITE};
            }
            bool d = ndp <= o.atol || (it > 0 && its == 0);
            if (!d && ndp_prev[r] >= 0) {
                const double rho = std::min(ndp / ndp_prev[r], 0.99);
                d = rho / (1.0 - rho) * ndp <= o.uzawa_tol * npn;
            }
            ndp_prev[r] = ndp;
            if (d) fin[r] = 1;
            else all = false;
        }
        if (fo.its >= o.max_it) conv = HDG_ERR_NOT_CONVERGED;
        if (all) break;
    }
    for (int r = 0; r < nrhs; ++r)
        if (!fin[r] && conv == HDG_OK) conv = HDG_ERR_NOT_CONVERGED;
    return conv;
}

} // namespace

// =====================================================================================
extern "C" {

void hdg_default_solve_opts(hdg_solve_opts *o) {
    if (!o) return;
    o->rtol = 1e-8;
    o->atol = 1e-10;
    o->floor_rel = 1e-10;
    o->krylov = 0;
    o->uzawa_tol = 1e-8;
    o->restart = 30;
    o->max_it = 1000;
    o->max_uzawa = 64;
}

const char *hdg_status_string(hdg_status s) {
    switch (s) {
    case HDG_OK: return "ok";
    case HDG_ERR_INVALID_ARG: return "invalid argument";
    case HDG_ERR_OOM: return "out of memory";
    case HDG_ERR_CUDA: return "CUDA error";
    case HDG_ERR_SINGULAR: return "singular factorisation";
    case HDG_ERR_NOT_CONVERGED: return "not converged";
    case HDG_ERR_BREAKDOWN: return "Krylov breakdown";
    case HDG_ERR_NONFINITE: return "non-finite value";
    case HDG_ERR_UNSUPPORTED: return "unsupported";
    case HDG_ERR_STATE: return "call order violated";
    case HDG_ERR_TIMEOUT: return "a bounded device wait timed out";
    }
    return "unknown status";
}

const char *hdg_last_error(const hdg_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

uint64_t hdg_kernel_launches(void) { return (uint64_t)launch_count(); }

int64_t hdg_reference_tables(int k, double *out) {
    if (k < 0 || k > MAX_K) return -1;
    try {
        RefTables t;
        build_reference_tables(k, t);
        int64_t n = 0;
        for (int i = 0; i < N_REF_TABLES; ++i) {
            const std::vector<double> *v = ref_table(t, i);
            if (out) std::memcpy(out + n, v->data(), sizeof(double) * v->size());
            n += (int64_t)v->size();
        }
        return n;
    } catch (...) {
        return -1;
    }
}

// topology, vertex patches and transfer tables of every level, on the host only;
// throws Fail{HDG_ERR_INVALID_ARG} (message in ctx->err) on an invalid hierarchy
void build_host_hierarchy(hdg_ctx *ctx, const hdg_mesh_desc *desc) {
    REQUIRE(desc->dim == 2, "dim must be 2 here");
    REQUIRE(desc->n_levels >= 1 && desc->n_levels <= MAX_LEVELS, "n_levels out of range 1..16");
    REQUIRE(desc->n_vertices && desc->n_cells && desc->coords && desc->cells, "null mesh arrays");
    const int nl = desc->n_levels;
    ctx->n_levels = nl;
    ctx->H.assign(nl, HostLevel());
    ctx->T.assign(nl, HostTransfer());
    for (int l = 0; l < nl; ++l) {
        HostLevel &H = ctx->H[l];
        H.nv = desc->n_vertices[l];
        H.nc = desc->n_cells[l];
        REQUIRE(H.nv >= 3 && H.nc >= 1 && H.nc < (1LL << 26), "level sizes out of range");
        REQUIRE(desc->coords[l] && desc->cells[l], "null level array");
        H.coords.assign(desc->coords[l], desc->coords[l] + 2 * H.nv);
        H.cells.assign(desc->cells[l], desc->cells[l] + 3 * H.nc);
        const int32_t *col = (desc->vertex_colour && desc->vertex_colour[l]) ? desc->vertex_colour[l] : nullptr;
        std::string e = build_level_topology(H, col);
        REQUIRE(e.empty(), "level " + std::to_string(l) + ": " + e);
        if (l > 0) {
            REQUIRE(desc->parent && desc->parent[l], "parent map required on levels >= 1");
            H.parent.assign(desc->parent[l], desc->parent[l] + H.nc);
            std::string e2 = build_transfer(ctx->H[l - 1], H, ctx->T[l]);
            REQUIRE(e2.empty(), "level " + std::to_string(l) + ": " + e2);
        }
    }
}

static void build_host_hierarchy_3d(hdg_ctx *ctx, const hdg_mesh_desc *desc);
static void upload_levels_3d(hdg_ctx *ctx);

hdg_status hdg_setup_mesh_hierarchy(const hdg_mesh_desc *desc, int device, hdg_ctx **out) {
    if (!out) return HDG_ERR_INVALID_ARG;
    *out = nullptr;
    if (!desc) return HDG_ERR_INVALID_ARG;
    hdg_ctx *ctx = new hdg_ctx();
    hdg_status st = guard(ctx, [&] {
        REQUIRE(desc->dim == 2 || desc->dim == 3, "dim must be 2 or 3");
        if (desc->dim == 3) build_host_hierarchy_3d(ctx, desc);
        else build_host_hierarchy(ctx, desc);
        const int nl = ctx->n_levels;
        ctx->L.resize(nl);
        // the hierarchy is valid (checked on the host, before any device call): upload
        int ndev = 0;
        CK(cudaGetDeviceCount(&ndev));
        REQUIRE(device >= 0 && device < ndev, "device ordinal out of range");
        ctx->device = device;
        CK(cudaSetDevice(device));
        if (ctx->dim == 3) upload_levels_3d(ctx);
        for (int l = 0; l < (ctx->dim == 2 ? nl : 0); ++l) {
            HostLevel &H = ctx->H[l];
            DevLevel &L = ctx->L[l];
            L.nv = H.nv;
            L.nc = H.nc;
            L.n_int = H.n_int;
            upload(ctx, L.coords, H.coords);
            upload(ctx, L.cells, H.cells);
            std::vector<int32_t> ci(3 * H.nc), fa(2 * H.n_int);
            for (int64_t c = 0; c < H.nc; ++c)
                for (int f = 0; f < 3; ++f) ci[3 * c + f] = H.interior_index[H.cell_facet[3 * c + f]];
            for (int64_t i = 0; i < H.n_int; ++i) {
                int F = H.interior_facets[i];
                for (int q = 0; q < 2; ++q) fa[2 * i + q] = (H.facet_cells[2 * F + q] << 2) | H.facet_lf[2 * F + q];
            }
            upload(ctx, L.cell_int, ci);
            if (l == nl - 1) {
                // boundary facets in facet order (inhomogeneous Dirichlet data of the finest level)
                std::vector<int32_t> bidx(H.nf, -1), cb(3 * H.nc, -1);
                int64_t nb = 0;
                for (int64_t F = 0; F < H.nf; ++F)
                    if (H.interior_index[F] < 0) bidx[F] = (int32_t)nb++;
                for (int64_t c = 0; c < H.nc; ++c)
                    for (int f = 0; f < 3; ++f) cb[3 * c + f] = bidx[H.cell_facet[3 * c + f]];
                L.n_bnd = nb;
                upload(ctx, L.cell_bnd, cb);
            }
            upload(ctx, L.facet_adj, fa);
            dalloc(ctx, L.cell_d, 3 * H.nc);
            dalloc(ctx, L.cell_area, H.nc);
            CK(launch_cell_geometry(L, 0));
            L.n_patches = H.n_patches;
            L.n_colours = H.n_colours;
            L.pf_max = H.pf_max;
            L.pc_max = H.pc_max;
            L.colour_ptr = H.colour_ptr;
            upload(ctx, L.patch_nf, H.patch_nf);
            upload(ctx, L.patch_facets, H.patch_facets);
            upload(ctx, L.patch_nc, H.patch_nc);
            upload(ctx, L.patch_cells, H.patch_cells);
            upload(ctx, L.patch_slot_src, H.patch_slot_src);
            if (l == nl - 1) {
                std::vector<int32_t> pci((size_t)H.n_patches * H.pc_max * 3, -1);
                for (int p = 0; p < H.n_patches; ++p)
                    for (int si = 0; si < H.patch_nc[p]; ++si) {
                        const int c = H.patch_cells[(size_t)p * H.pc_max + si];
                        for (int f = 0; f < 3; ++f) pci[((size_t)p * H.pc_max + si) * 3 + f] = ci[3 * c + f];
                    }
                upload(ctx, L.patch_cint, pci);
                upload(ctx, L.patch_cext, H.patch_cext);
            }
            {
                // the two vertex-patch slots of every interior facet (block Jacobi gather)
                std::vector<int32_t> fs(2 * H.n_int, -1);
                for (int p = 0; p < H.n_patches; ++p)
                    for (int js = 0; js < H.patch_nf[p]; ++js) {
                        const int F = H.patch_facets[(size_t)p * H.pf_max + js];
                        const int q = fs[2 * F] < 0 ? 0 : 1;
                        fs[2 * F + q] = p * H.pf_max + js;
                    }
                upload(ctx, L.facet_slot, fs);
            }
            if (H.nc <= GS0_TABLE_MAX_CELLS && 2 * H.pf_max <= 16) {
                // lowest-order gather table: each lane of the sweep reads its row's whole
                // gather pattern at once instead of chasing patch -> cell -> facet indices
                const int npm = 2 * H.pf_max;
                std::vector<int32_t> tb((size_t)H.n_patches * npm * GS0_TABLE_INTS, -1);
                for (int p = 0; p < H.n_patches; ++p)
                    for (int t = 0; t < 2 * H.patch_nf[p]; ++t) {
                        int32_t *e = &tb[((size_t)p * npm + t) * GS0_TABLE_INTS];
                        const int js = t >> 1, d = t & 1;
                        e[0] = 2 * H.patch_facets[(size_t)p * H.pf_max + js] + d;
                        for (int q = 0; q < 2; ++q) {
                            const int src = H.patch_slot_src[((size_t)p * H.pf_max + js) * 2 + q];
                            const int c = H.patch_cells[(size_t)p * H.pc_max + (src >> 2)];
                            e[1 + q] = c * 36 + (src & 3) * 12 + d;
                            for (int f2 = 0; f2 < 3; ++f2) e[3 + 3 * q + f2] = ci[3 * c + f2];
                        }
                    }
                upload(ctx, L.gs0_table, tb);
            }
            if (l > 0) {
                HostTransfer &T = ctx->T[l];
                L.nc_coarse = T.nc_coarse;
                L.nB = T.nB;
                upload(ctx, L.tr_slots, T.slots);
                upload(ctx, L.tr_nbr, T.nbr);
                upload(ctx, L.tr_children, T.children);
                upload(ctx, L.tr_child_slot, T.child_slot);
                upload(ctx, L.tr_fineB, T.fineB);
                upload(ctx, L.tr_fineB_src, T.fineB_src);
                upload(ctx, L.tr_W, T.W);
                std::vector<float> Wf(T.W.begin(), T.W.end());
                upload(ctx, L.tr_Wf, Wf);
                dalloc(ctx, L.tr_H, 72 * T.nc_coarse);
                dalloc(ctx, L.tr_Hf, 72 * T.nc_coarse);
                dalloc(ctx, L.ct1, 12 * T.nc_coarse);
                dalloc(ctx, L.ct2, 6 * T.nc_coarse);
                dalloc(ctx, L.ct1f, 12 * T.nc_coarse);
                dalloc(ctx, L.ct2f, 6 * T.nc_coarse);
            }
            const int64_t n0 = std::max<int64_t>(2 * H.n_int, 1);
            dalloc(ctx, L.g, n0); dalloc(ctx, L.u, n0); dalloc(ctx, L.r, n0); dalloc(ctx, L.t, n0);
            dalloc(ctx, L.gf, n0); dalloc(ctx, L.uf, n0); dalloc(ctx, L.rf, n0); dalloc(ctx, L.tf, n0);
        }
        dalloc(ctx, ctx->status_flag, 1);
        dalloc(ctx, ctx->wait_flag, 1);
        CK(cudaMemset(ctx->wait_flag.p, 0, sizeof(int)));
        CK(cudaMallocHost((void **)&ctx->h_pinned, 8 * sizeof(double)));
        CK(cudaDeviceSynchronize());
    });
    if (st != HDG_OK) {
        // keep the message reachable through a minimal context
        *out = ctx;
        return st;
    }
    *out = ctx;
    return HDG_OK;
}

hdg_status hdg_check_hierarchy(const hdg_mesh_desc *desc, int k, hdg_hierarchy_info *info, char *msg,
                               int msg_len) {
    if (msg && msg_len > 0) msg[0] = 0;
    if (!desc) return HDG_ERR_INVALID_ARG;
    hdg_ctx tmp;
    hdg_ctx *ctx = &tmp;
    hdg_status st = guard(ctx, [&] {
        if (desc->dim == 3) {
            REQUIRE(k >= 0 && k <= MAX_K3, "3D: k out of range 0..3");
            build_host_hierarchy_3d(ctx, desc);
            if (info) {
                const HostLevel3 &F = ctx->H3[ctx->n_levels - 1];
                info->n_levels = ctx->n_levels;
                info->n_interior_facets = F.n_int;
                info->n_dof = (int64_t)F.n_int * dpf3(k);
                info->n_patches = F.n_patches;
                info->n_colours = F.n_colours;
                info->max_patch_facets = F.pf_max;
                info->max_patch_cells = F.pc_max;
            }
            return;
        }
        REQUIRE(k >= 0 && k <= 4, "k out of range 0..4");
        build_host_hierarchy(ctx, desc);
        if (info) {
            const HostLevel &F = ctx->H[ctx->n_levels - 1];
            info->n_levels = ctx->n_levels;
            info->n_interior_facets = F.n_int;
            info->n_dof = (int64_t)F.n_int * 2 * (k + 1);
            info->n_patches = F.n_patches;
            info->n_colours = F.n_colours;
            info->max_patch_facets = F.pf_max;
            info->max_patch_cells = F.pc_max;
        }
    });
    if (st != HDG_OK && msg && msg_len > 0) {
        std::strncpy(msg, tmp.err.c_str(), (size_t)msg_len - 1);
        msg[msg_len - 1] = 0;
    }
    return st;
}

void hdg_destroy(hdg_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    for (auto &L : ctx->L) free_level(L);
    free_operator(ctx->opk);
    dfree(ctx->refk_dev); dfree(ctx->ref0_dev);
    dfree(ctx->kr); dfree(ctx->ku); dfree(ctx->kt); dfree(ctx->krf); dfree(ctx->kuf); dfree(ctx->kgf);
    dfree(ctx->post_tabs); dfree(ctx->pcg_buf); dfree(ctx->jD); dfree(ctx->jDf); dfree(ctx->dir_x);
    dfree(ctx->dir_flux); dfree(ctx->pic_f);
    dfree(ctx->coarse_inv); dfree(ctx->status_flag); dfree(ctx->wait_flag); dfree(ctx->conv_k); dfree(ctx->newton_x);
    dfree(ctx->V); dfree(ctx->Z); dfree(ctx->w); dfree(ctx->partials); dfree(ctx->small);
    dfree(ctx->uz_partials);
    for (auto *b : {&ctx->rec_L, &ctx->rec_La, &ctx->rec_rt, &ctx->rec_ulat, &ctx->rec_e, &ctx->rec_j, &ctx->adj_F,
                    &ctx->adj_u, &ctx->adj_p, &ctx->pic_F, &ctx->pic_w0, &ctx->pic_w1, &ctx->pic_e, &ctx->pic_j,
                    &ctx->pic_x})
        dfree(*b);
    drop_graph(ctx);
    dfree(ctx->pc_in); dfree(ctx->pc_out);
    for (auto *b : {&ctx->mV, &ctx->mZ, &ctx->mw, &ctx->mpart, &ctx->msmall, &ctx->mhbuf, &ctx->mF, &ctx->mU,
                    &ctx->mP, &ctx->mG, &ctx->mkr, &ctx->mkt, &ctx->mrd, &ctx->mzd, &ctx->pcm_in, &ctx->pcm_out})
        dfree(*b);
    dfree(ctx->mkgf); dfree(ctx->mkuf); dfree(ctx->mkrf); dfree(ctx->mint); dfree(ctx->mxs); dfree(ctx->tune_buf);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->batch_stream) cudaStreamDestroy(ctx->batch_stream);
    if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
    if (ctx->h_multi) cudaFreeHost(ctx->h_multi);
    delete ctx;
}

hdg_status hdg_get_sizes(const hdg_ctx *cctx, hdg_sizes *out) {
    if (!cctx || !out) return HDG_ERR_INVALID_ARG;
    std::memset(out, 0, sizeof(*out));
    const hdg_ctx *ctx = cctx;
    if (ctx->n_levels < 1) return HDG_ERR_STATE;
    if (ctx->dim == 3) {
        const HostLevel3 &H = ctx->H3[ctx->n_levels - 1];
        const int k = ctx->prm.k;
        out->k = ctx->condensed ? k : -1;
        out->n_levels = ctx->n_levels;
        out->n_cells = H.nc;
        out->n_interior_facets = H.n_int;
        out->n_dof = ctx->condensed ? ctx->n_dof : 0;
        for (int l = 0; l < ctx->n_levels; ++l) {
            out->n_dof_level[l] = 3 * ctx->H3[l].n_int;
            out->n_colours_level[l] = ctx->H3[l].n_colours;
        }
        out->n_lat = ctx->condensed ? (k + 2) * (k + 3) * (k + 4) / 6 : 0;
        out->n_boundary_facets = H.nf - H.n_int;
        return HDG_OK;
    }
    const HostLevel &H = ctx->H[ctx->n_levels - 1];
    out->k = ctx->condensed ? ctx->prm.k : -1;
    out->n_levels = ctx->n_levels;
    out->n_cells = H.nc;
    out->n_interior_facets = H.n_int;
    out->n_dof = ctx->condensed ? ctx->n_dof : 0;
    for (int l = 0; l < ctx->n_levels; ++l) {
        out->n_dof_level[l] = 2 * ctx->H[l].n_int;
        out->n_colours_level[l] = ctx->H[l].n_colours;
    }
    out->n_lat = ctx->condensed ? (ctx->prm.k + 2) * (ctx->prm.k + 3) / 2 : 0;
    out->n_boundary_facets = H.nf - H.n_int;
    return HDG_OK;
}

hdg_status hdg_boundary_facets(const hdg_ctx *ctx, int32_t *pairs) {
    if (!ctx || !pairs) return HDG_ERR_INVALID_ARG;
    if (ctx->n_levels < 1) return HDG_ERR_STATE;
    if (ctx->dim == 3) {
        const HostLevel3 &H = ctx->H3[ctx->n_levels - 1];
        int64_t b = 0;
        for (int64_t F = 0; F < H.nf; ++F)
            if (H.interior_index[F] < 0) {
                for (int q = 0; q < 3; ++q) pairs[3 * b + q] = H.face_v[3 * F + q];
                ++b;
            }
        return HDG_OK;
    }
    const HostLevel &H = ctx->H[ctx->n_levels - 1];
    int64_t b = 0;
    for (int64_t F = 0; F < H.nf; ++F)
        if (H.interior_index[F] < 0) {
            pairs[2 * b] = H.facet_v[2 * F];
            pairs[2 * b + 1] = H.facet_v[2 * F + 1];
            ++b;
        }
    return HDG_OK;
}

static void upload_ref(hdg_ctx *ctx, RefTables &t, DBuf<double> &d, int k) {
    if (t.k == k && d.p) return;
    build_reference_tables(k, t);
    std::vector<double> packed;
    for (int i = 0; i < N_REF_TABLES; ++i) {
        const std::vector<double> *v = ref_table(t, i);
        packed.insert(packed.end(), v->begin(), v->end());
    }
    dfree(d);
    upload(ctx, d, packed);
}

// Element matrices, patch inverses, transfer blocks and the coarsest inverse of
// every level from ctx->prm (and ctx->conv_k / ctx->conv_t for Oseen); the
// order-k element loads of `forcing` (NULL = zero).

// the FP32 closed-form sweeps' augmented-Lagrangian split (op.swQ, op.swA00) on the 2D level
// with the outside-facet table, for the FP32 preconditioners; returns whether it was allocated
static bool alloc_al_split(hdg_ctx *ctx, const DevLevel &L, DevOperator &op) {
    if (ctx->prm.precision == HDG_FP64 || !L.patch_cext.p || L.n_patches == 0) {
        dfree(op.swQ);
        dfree(op.swA00);
        return false;
    }
    dalloc(ctx, op.swQ, (size_t)L.n_patches * L.pc_max * op.np_max);
    dalloc(ctx, op.swA00, (size_t)L.n_patches * L.pf_max * 2);
    return true;
}

static void condense_all(hdg_ctx *ctx, const double *forcing, cudaStream_t s) {
    const hdg_params *prm = &ctx->prm;
    ctx->condensed = false;
    drop_graph(ctx);
    std::memset(ctx->tile_rb, 0, sizeof ctx->tile_rb);   // a new operator is tuned afresh
    std::memset(ctx->tile_nt, 0, sizeof ctx->tile_nt);
    std::memset(ctx->tile_ms, 0, sizeof ctx->tile_ms);
    std::memset(ctx->tile_tc_nt, 0, sizeof ctx->tile_tc_nt);
    std::memset(ctx->tile_tc_ms, 0, sizeof ctx->tile_tc_ms);
    const int k = prm->k;
    upload_ref(ctx, ctx->ref0, ctx->ref0_dev, 0);
    upload_ref(ctx, ctx->refk, ctx->refk_dev, k);
    CK(cudaMemsetAsync(ctx->status_flag.p, 0, sizeof(int), s));
    const int nl = ctx->n_levels;
    const bool per_cell = prm->nu_elem != nullptr;
    if (ctx->has_conv) {
        // RT_0 convecting fields of the lowest-order levels from the finest field's fluxes
        DevLevel &F = ctx->L[nl - 1];
        dalloc(ctx, F.conv_flux, 3 * F.nc);
        CK(launch_conv_flux(F, ctx->refk_dev.p, ctx->refk, ctx->conv_k.p, F.conv_flux.p, s));
        for (int l = nl - 1; l >= 1; --l) {
            dalloc(ctx, ctx->L[l - 1].conv_flux, 3 * ctx->L[l - 1].nc);
            CK(launch_flux_restrict(ctx->L[l], ctx->L[l].conv_flux.p, ctx->L[l - 1].conv_flux.p, s));
        }
        for (int l = 0; l < nl; ++l) {
            dalloc(ctx, ctx->L[l].conv_lat, 6 * ctx->L[l].nc);
            CK(launch_rt0_vertex(ctx->L[l], ctx->L[l].conv_flux.p, ctx->L[l].conv_lat.p, s));
        }
    }
    for (int l = 0; l < nl; ++l) {
        DevLevel &L = ctx->L[l];
        DevOperator &op = L.op0;
        op.k = 0; op.dpf = 2; op.nloc = 6; op.np_max = L.pf_max * 2;
        dalloc(ctx, op.A, 36 * L.nc);
        dalloc(ctx, op.Af, 36 * L.nc);
        dalloc(ctx, op.Pinv, (size_t)L.n_patches * op.np_max * op.np_max);
        dalloc(ctx, op.Pinvf, (size_t)L.n_patches * op.np_max * op.np_max);
        CK(launch_condense(0, L, ctx->ref0_dev.p, ctx->ref0, prm->nu, per_cell ? L.cell_nu.p : nullptr,
                           prm->beta, prm->gamma, nullptr, ctx->has_conv ? L.conv_lat.p : nullptr, ctx->conv_t,
                           nullptr, op.A.p, op.Af.p, nullptr, ctx->status_flag.p, RecoverArgs(), s));
        CK(launch_patch_inverse(L, op, ctx->has_conv ? 1 : 0, ctx->status_flag.p, s));
    }
    DevLevel &LJ = ctx->L[nl - 1];
    DevOperator &op = ctx->opk;
    op.k = k; op.dpf = 2 * (k + 1); op.nloc = 3 * op.dpf; op.np_max = LJ.pf_max * op.dpf;
    op.alo_valid = false;
    dalloc(ctx, op.A, (size_t)op.nloc * op.nloc * LJ.nc);
    dalloc(ctx, op.Af, (size_t)op.nloc * op.nloc * LJ.nc);
    dalloc(ctx, op.Fel, (size_t)op.nloc * LJ.nc);
    dalloc(ctx, op.Pinv, (size_t)LJ.n_patches * op.np_max * op.np_max);
    dalloc(ctx, op.Pinvf, (size_t)LJ.n_patches * op.np_max * op.np_max);
    CK(launch_condense(k, LJ, ctx->refk_dev.p, ctx->refk, prm->nu, per_cell ? LJ.cell_nu.p : nullptr,
                       prm->beta, prm->gamma, forcing, conv_of(ctx), ctx->conv_t, newton_of(ctx), op.A.p, op.Af.p,
                       op.Fel.p, ctx->status_flag.p, RecoverArgs(), s));
    CK(launch_patch_inverse(LJ, op, ctx->has_conv ? 1 : 0, ctx->status_flag.p, s));
    if (alloc_al_split(ctx, LJ, op))
        CK(launch_al_split(LJ, op, prm->nu, per_cell ? LJ.cell_nu.p : nullptr, prm->gamma, s));
    op.tma_flag = ctx->wait_flag.p;
    if (!ctx->has_conv && k >= 1 && prm->precision != HDG_FP64) {
        // symmetric patch inverses: the FP32 sweep reads packed triangles (half the bytes)
        dalloc(ctx, op.Pinvp, (size_t)LJ.n_patches * packed_patch_size(op.np_max));
        CK(launch_pack_sym(LJ, op, s));
    } else {
        dfree(op.Pinvp);
    }
    op.h_fmt = 0;
    if (k >= 1 && (prm->precision == HDG_MIXED_BF16 || prm->precision == HDG_MIXED_FP16)) {
        dalloc(ctx, op.Ah, (size_t)op.nloc * op.nloc * LJ.nc);
        dalloc(ctx, op.Ah_s, (size_t)op.nloc * LJ.nc);
        dalloc(ctx, op.Pinvh, (size_t)LJ.n_patches * op.np_max * op.np_max);
        dalloc(ctx, op.Pinvh_s, (size_t)LJ.n_patches * op.np_max);
        CK(launch_round16(LJ, op, (int)prm->precision, s));
        op.h_fmt = (int)prm->precision;
    }
    for (int l = 1; l < nl; ++l) CK(launch_transfer_H(ctx->L[l], ctx->status_flag.p, s));
    ctx->n0 = 2 * ctx->L[0].n_int;
    dalloc(ctx, ctx->coarse_inv, std::max<int64_t>(ctx->n0 * ctx->n0, 1));
    CK(launch_coarse_inverse(ctx->L[0], ctx->coarse_inv.p, ctx->n0, ctx->status_flag.p, s));
    ctx->small_Ls = prm->smoother == 1 ? -1 : small_levels(ctx);   // the fused kernel sweeps by GS
    if (prm->smoother == 1) {
        size_t nd = (size_t)LJ.n_patches * op.np_max;
        for (int l = 0; l < nl; ++l) nd = std::max(nd, (size_t)ctx->L[l].n_patches * ctx->L[l].op0.np_max);
        dalloc(ctx, ctx->jD, std::max<size_t>(nd, 1));
        dalloc(ctx, ctx->jDf, std::max<size_t>(nd, 1));
    }
    if (ctx->small_Ls >= 1) {
        const size_t cb_d = fill_small<double>(ctx, ctx->small_Ls);
        const size_t cb_f = fill_small<float>(ctx, ctx->small_Ls);
        int npm = 2;
        for (int l = 1; l <= ctx->small_Ls; ++l) npm = std::max(npm, ctx->L[l].op0.np_max);
        ctx->small_cs_d = mg_small_cluster_size<double>(cb_d, npm * (int)sizeof(double));
        ctx->small_cs_f = mg_small_cluster_size<float>(cb_f, npm * (int)sizeof(float));
        ctx->small_smem_d = mg_small_smem(cb_d, std::max(ctx->small_cs_d, 1), npm * (int)sizeof(double));
        ctx->small_smem_f = mg_small_smem(cb_f, std::max(ctx->small_cs_f, 1), npm * (int)sizeof(float));
        // a single block keeps all level vectors in its shared memory when they fit
        if (ctx->small_cs_d == 1) make_resident(ctx->small_d, ctx->small_Ls, ctx->small_smem_d);
        if (ctx->small_cs_f == 1) make_resident(ctx->small_f, ctx->small_Ls, ctx->small_smem_f);
        if (ctx->small_cs_d == 0 || ctx->small_cs_f == 0) ctx->small_Ls = -1;
    }
    ctx->n_dof = LJ.n_int * op.dpf;
    const int64_t nd = std::max<int64_t>(ctx->n_dof, 1);
    dalloc(ctx, ctx->kr, nd); dalloc(ctx, ctx->ku, nd); dalloc(ctx, ctx->kt, nd);
    dalloc(ctx, ctx->krf, nd); dalloc(ctx, ctx->kuf, nd); dalloc(ctx, ctx->kgf, nd);
    check_flag(ctx, s);
    ctx->condensed = true;
}

// ===================================================================== 3D (tetrahedra)
// The 3D path shares the context, the device levels, the Krylov and Uzawa drivers and the
// multigrid recursion with 2D; these functions build its host topology, upload it and
// condense its operators (condense3d.cu, topology3d.cpp, reference3d.cpp).

static void build_host_hierarchy_3d(hdg_ctx *ctx, const hdg_mesh_desc *desc) {
    REQUIRE(desc->n_levels >= 1 && desc->n_levels <= MAX_LEVELS, "n_levels out of range 1..16");
    REQUIRE(desc->n_vertices && desc->n_cells && desc->coords && desc->cells, "null mesh arrays");
    const int nl = desc->n_levels;
    ctx->dim = 3;
    ctx->n_levels = nl;
    ctx->H3.assign(nl, HostLevel3());
    ctx->T3.assign(nl, HostTransfer3());
    for (int l = 0; l < nl; ++l) {
        HostLevel3 &H = ctx->H3[l];
        H.nv = desc->n_vertices[l];
        H.nc = desc->n_cells[l];
        REQUIRE(H.nv >= 4 && H.nc >= 1 && H.nc < (1LL << 26), "level sizes out of range");
        REQUIRE(desc->coords[l] && desc->cells[l], "null level array");
        H.coords.assign(desc->coords[l], desc->coords[l] + 3 * H.nv);
        H.cells.assign(desc->cells[l], desc->cells[l] + 4 * H.nc);
        std::string e = build_level_topology_3d(H);
        REQUIRE(e.empty(), "level " + std::to_string(l) + ": " + e);
        if (l > 0) {
            REQUIRE(desc->parent && desc->parent[l], "parent map required on levels >= 1");
            H.parent.assign(desc->parent[l], desc->parent[l] + H.nc);
            std::string e2 = build_transfer_3d(ctx->H3[l - 1], H, ctx->T3[l]);
            REQUIRE(e2.empty(), "level " + std::to_string(l) + ": " + e2);
        }
    }
}

static void upload_levels_3d(hdg_ctx *ctx) {
    for (int l = 0; l < ctx->n_levels; ++l) {
        HostLevel3 &H = ctx->H3[l];
        DevLevel &L = ctx->L[l];
        L.dim = 3;
        L.nv = H.nv;
        L.nc = H.nc;
        L.n_int = H.n_int;
        upload(ctx, L.coords, H.coords);
        upload(ctx, L.cells, H.cells);
        std::vector<int32_t> ci(4 * H.nc), fa(2 * H.n_int);
        for (int64_t c = 0; c < 4 * H.nc; ++c) ci[c] = H.interior_index[H.cell_face[c]];
        for (int64_t i = 0; i < H.n_int; ++i) {
            const int F = H.interior_faces[i];
            for (int q = 0; q < 2; ++q) fa[2 * i + q] = (H.face_cells[2 * F + q] << 2) | H.face_lf[2 * F + q];
        }
        upload(ctx, L.cell_int, ci);
        upload(ctx, L.facet_adj, fa);
        L.n_bnd = H.nf - H.n_int;
        if (l == ctx->n_levels - 1) {
            // boundary faces in face order (inhomogeneous Dirichlet data of the finest level)
            std::vector<int32_t> bidx(H.nf, -1), cb(4 * H.nc, -1);
            int64_t nb = 0;
            for (int64_t F = 0; F < H.nf; ++F)
                if (H.interior_index[F] < 0) bidx[F] = (int32_t)nb++;
            for (int64_t c = 0; c < 4 * H.nc; ++c) cb[c] = bidx[H.cell_face[c]];
            upload(ctx, L.cell_bnd, cb);
        }
        dalloc(ctx, L.cell_d, 4 * H.nc);
        dalloc(ctx, L.cell_area, H.nc);
        L.n_patches = H.n_patches;
        L.n_colours = H.n_colours;
        L.pf_max = H.pf_max;
        L.pc_max = H.pc_max;
        L.colour_ptr = H.colour_ptr;
        upload(ctx, L.patch_nf, H.patch_nf);
        upload(ctx, L.patch_facets, H.patch_facets);
        upload(ctx, L.patch_nc, H.patch_nc);
        upload(ctx, L.patch_cells, H.patch_cells);
        upload(ctx, L.patch_slot_src, H.patch_slot_src);
        upload(ctx, L.patch_cext, H.patch_cext);
        if (l > 0) {
            HostTransfer3 &T = ctx->T3[l];
            L.nc_coarse = T.nc_coarse;
            L.nB = T.nB;
            upload(ctx, L.tr_slots, T.slots);
            upload(ctx, L.tr_nbr, T.nbr);
            upload(ctx, L.tr_children, T.children);
            upload(ctx, L.tr_child_slot, T.child_slot);
            upload(ctx, L.tr_fineB, T.fineB);
            upload(ctx, L.tr_fineB_src, T.fineB_src);
            upload(ctx, L.tr_W, T.W);
            std::vector<float> Wf(T.W.begin(), T.W.end());
            upload(ctx, L.tr_Wf, Wf);
            const size_t nh = (size_t)3 * TR3_T * 3 * TR3_B * T.nc_coarse;
            dalloc(ctx, L.tr_H, nh);
            dalloc(ctx, L.tr_Hf, nh);
            dalloc(ctx, L.ct1, 3 * TR3_B * T.nc_coarse);
            dalloc(ctx, L.ct2, 12 * T.nc_coarse);
            dalloc(ctx, L.ct1f, 3 * TR3_B * T.nc_coarse);
            dalloc(ctx, L.ct2f, 12 * T.nc_coarse);
        }
        const int64_t n0 = std::max<int64_t>(3 * H.n_int, 1);
        dalloc(ctx, L.g, n0); dalloc(ctx, L.u, n0); dalloc(ctx, L.r, n0); dalloc(ctx, L.t, n0);
        dalloc(ctx, L.gf, n0); dalloc(ctx, L.uf, n0); dalloc(ctx, L.rf, n0); dalloc(ctx, L.tf, n0);
    }
}

static void upload_ref3(hdg_ctx *ctx, RefTables3 &t, DBuf<double> &d, int k) {
    if (t.k == k && d.p) return;
    build_reference_tables_3d(k, t);
    dfree(d);
    upload(ctx, d, pack_reference_tables_3d(t));
}

static int condense3_blocks(hdg_ctx *ctx) {
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
    return 2 * std::max(sms, 1);
}

static void condense_all_3d(hdg_ctx *ctx, const double *forcing, cudaStream_t s) {
    const hdg_params *prm = &ctx->prm;
    ctx->condensed = false;
    drop_graph(ctx);
    const int k = prm->k;
    upload_ref3(ctx, ctx->ref30, ctx->ref30_dev, 0);
    upload_ref3(ctx, ctx->ref3k, ctx->ref3k_dev, k);
    CK(cudaMemsetAsync(ctx->status_flag.p, 0, sizeof(int), s));
    const int nl = ctx->n_levels, blocks = condense3_blocks(ctx);
    {
        // one workspace for the condensation and the patch inverses, sized before any launch
        size_t need = condense3_scratch_doubles(k, blocks);
        for (int l = 0; l < nl; ++l) {
            const int npm = ctx->L[l].pf_max * (l == nl - 1 ? dpf3(k) : 3);
            need = std::max(need, (size_t)std::min(std::max(ctx->L[l].n_patches, 1), blocks) * npm * npm);
        }
        dalloc(ctx, ctx->c3_scratch, need);
    }
    int *flag = ctx->status_flag.p;
    for (int l = 0; l < nl; ++l) {
        DevLevel &L = ctx->L[l];
        DevOperator &op = L.op0;
        op.k = 0; op.dpf = 3; op.nloc = 12; op.np_max = L.pf_max * 3;
        dalloc(ctx, op.A, 144 * L.nc);
        dalloc(ctx, op.Af, 144 * L.nc);
        dalloc(ctx, op.Pinv, (size_t)L.n_patches * op.np_max * op.np_max);
        dalloc(ctx, op.Pinvf, (size_t)L.n_patches * op.np_max * op.np_max);
        CK(launch_condense3(0, L, ctx->ref30_dev.p, ctx->ref30, prm->nu, nullptr, prm->beta, prm->gamma, nullptr,
                            op.A.p, op.Af.p, nullptr, ctx->c3_scratch.p, blocks, flag, s));
        CK(launch_patch_inverse3(L, op, ctx->c3_scratch.p, blocks, flag, s));
    }
    DevLevel &LJ = ctx->L[nl - 1];
    DevOperator &op = ctx->opk;
    op.k = k; op.dpf = dpf3(k); op.nloc = 4 * op.dpf; op.np_max = LJ.pf_max * op.dpf;
    op.alo_valid = false;
    dalloc(ctx, op.A, (size_t)op.nloc * op.nloc * LJ.nc);
    dalloc(ctx, op.Af, (size_t)op.nloc * op.nloc * LJ.nc);
    dalloc(ctx, op.Fel, (size_t)op.nloc * LJ.nc);
    // the FP32 preconditioner sweeps with the FP32 inverses only: no FP64 copy is kept (at n = 48, k = 3
    // the FP64 edge-patch inverses alone would take about 200 GB)
    if (prm->precision == HDG_FP64) dalloc(ctx, op.Pinv, (size_t)LJ.n_patches * op.np_max * op.np_max);
    else dfree(op.Pinv);
    dalloc(ctx, op.Pinvf, (size_t)LJ.n_patches * op.np_max * op.np_max);
    CK(launch_condense3(k, LJ, ctx->ref3k_dev.p, ctx->ref3k, prm->nu, nullptr, prm->beta, prm->gamma, forcing, op.A.p,
                        op.Af.p, op.Fel.p, ctx->c3_scratch.p, blocks, flag, s));
    CK(launch_patch_inverse3(LJ, op, ctx->c3_scratch.p, blocks, flag, s));
    op.tma_flag = nullptr;
    dfree(op.Pinvp);   // full transposed inverses: the packed form staged in shared memory measured 3.2x slower
    op.h_fmt = 0;
    for (int l = 1; l < nl; ++l) CK(launch_transfer_H3(ctx->L[l], flag, s));
    ctx->n0 = 3 * ctx->L[0].n_int;
    dalloc(ctx, ctx->coarse_inv, std::max<int64_t>(ctx->n0 * ctx->n0, 1));
    CK(launch_coarse_inverse(ctx->L[0], ctx->coarse_inv.p, ctx->n0, flag, s));
    ctx->small_Ls = -1;
    ctx->n_dof = LJ.n_int * op.dpf;
    const int64_t nd = std::max<int64_t>(ctx->n_dof, 1);
    dalloc(ctx, ctx->kr, nd); dalloc(ctx, ctx->ku, nd); dalloc(ctx, ctx->kt, nd);
    dalloc(ctx, ctx->krf, nd); dalloc(ctx, ctx->kuf, nd); dalloc(ctx, ctx->kgf, nd);
    check_flag(ctx, s);
    ctx->condensed = true;
}

static void condense_3d(hdg_ctx *ctx, const hdg_params *prm, const double *forcing, double *rhs_out,
                        cudaStream_t s) {
    REQUIRE(prm->k >= 0 && prm->k <= MAX_K3, "3D: k out of range 0..3");
    REQUIRE(prm->nu > 0 && std::isfinite(prm->nu), "nu must be positive");
    REQUIRE(prm->beta >= 0 && std::isfinite(prm->beta), "beta must be >= 0");
    REQUIRE(prm->gamma >= 0 && std::isfinite(prm->gamma), "gamma must be >= 0");
    REQUIRE(prm->m_p >= 1 && prm->m_h >= 1, "m_p, m_h must be >= 1");
    REQUIRE(prm->cycle == 1 || prm->cycle == 2, "cycle must be 1 (V) or 2 (W)");
    REQUIRE(prm->vcycle_growth >= 1 && prm->vcycle_growth <= 4, "vcycle_growth out of range 1..4");
    REQUIRE(prm->hp_additive == 0 || prm->hp_additive == 1, "hp_additive must be 0 or 1");
    if (!(prm->precision == HDG_FP64 || prm->precision == HDG_MIXED_FP32) || prm->smoother != 0 ||
        prm->fused_coarse_cells != 0 || prm->nu_elem || prm->conv || prm->newton_u) {
        ctx->err = "3D supports the generalized Stokes operator with a scalar viscosity, Dirichlet data, block GS "
                   "and the FP64 or FP32 preconditioner";
        throw Fail{HDG_ERR_UNSUPPORTED};
    }
    REQUIRE(3 * ctx->L[0].n_int <= MAX_COARSE_DOFS,
            "coarsest level has " + std::to_string(3 * ctx->L[0].n_int) +
                " unknowns; the dense coarse solve allows at most " + std::to_string(MAX_COARSE_DOFS));
    ctx->prm = *prm;
    ctx->has_conv = ctx->has_newton = false;
    condense_all_3d(ctx, forcing, s);
    // inhomogeneous Dirichlet data: a copy, the cells' boundary fluxes and the load coupling
    DevLevel &LJ = ctx->L[ctx->n_levels - 1];
    ctx->has_dir = prm->dirichlet != nullptr;
    if (ctx->has_dir) {
        const size_t nb = (size_t)LJ.n_bnd * dpf3(prm->k);
        dalloc(ctx, ctx->dir_x, std::max<size_t>(nb, 1));
        CK(cudaMemcpyAsync(ctx->dir_x.p, prm->dirichlet, sizeof(double) * nb, cudaMemcpyDeviceToDevice, s));
        dalloc(ctx, ctx->dir_flux, std::max<int64_t>(LJ.nc, 1));
        CK(launch_boundary_flux(LJ, dpf3(prm->k), ctx->dir_x.p, ctx->dir_flux.p, s));
    }
    if (rhs_out) {
        if (forcing) CK(launch_assemble_load(LJ, ctx->opk, rhs_out, s));
        else CK(cudaMemsetAsync(rhs_out, 0, sizeof(double) * ctx->n_dof, s));
        if (ctx->has_dir) CK(launch_dirichlet_load(LJ, ctx->opk, ctx->dir_x.p, rhs_out, s));
    }
}

hdg_status hdg_condense(hdg_ctx *ctx, const hdg_params *prm, const double *forcing, double *rhs_out,
                        hdg_stream_t stream) {
    if (!ctx) return HDG_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        REQUIRE(prm, "null params");
        if (ctx->dim == 3) {
            CK(cudaSetDevice(ctx->device));
            condense_3d(ctx, prm, forcing, rhs_out, (cudaStream_t)stream);
            return;
        }
        REQUIRE(prm->k >= 0 && prm->k <= MAX_K, "k out of range 0..4");
        REQUIRE(prm->nu > 0 && std::isfinite(prm->nu), "nu must be positive");
        REQUIRE(prm->beta >= 0 && std::isfinite(prm->beta), "beta must be >= 0");
        REQUIRE(prm->gamma >= 0 && std::isfinite(prm->gamma), "gamma must be >= 0");
        REQUIRE(prm->m_p >= 1 && prm->m_h >= 1, "m_p, m_h must be >= 1");
        REQUIRE(prm->cycle == 1 || prm->cycle == 2, "cycle must be 1 (V) or 2 (W)");
        REQUIRE(prm->vcycle_growth >= 1 && prm->vcycle_growth <= 4, "vcycle_growth out of range 1..4");
        REQUIRE(prm->precision == HDG_FP64 || prm->precision == HDG_MIXED_FP32 ||
                    prm->precision == HDG_MIXED_BF16 || prm->precision == HDG_MIXED_FP16, "unknown precision");
        REQUIRE(prm->fused_coarse_cells >= 0, "fused_coarse_cells must be >= 0");
        REQUIRE(prm->smoother == 0 || prm->smoother == 1, "smoother must be 0 (block GS) or 1 (block Jacobi)");
        REQUIRE(std::isfinite(prm->jacobi_damping) && prm->jacobi_damping < 2, "jacobi_damping out of range");
        REQUIRE(prm->hp_additive == 0 || prm->hp_additive == 1, "hp_additive must be 0 or 1");
        REQUIRE(2 * ctx->L[0].n_int <= MAX_COARSE_DOFS,
                "coarsest level has " + std::to_string(2 * ctx->L[0].n_int) +
                " unknowns; the dense coarse solve allows at most " + std::to_string(MAX_COARSE_DOFS) +
                " (add coarser levels)");
        CK(cudaSetDevice(ctx->device));
        cudaStream_t s = (cudaStream_t)stream;
        ctx->condensed = false;
        ctx->prm = *prm;
        const int nl = ctx->n_levels;
        // per-cell viscosity: the caller's on the finest level, child means below
        if (prm->nu_elem) {
            DevLevel &F = ctx->L[nl - 1];
            dalloc(ctx, F.cell_nu, F.nc);
            CK(cudaMemcpyAsync(F.cell_nu.p, prm->nu_elem, sizeof(double) * F.nc, cudaMemcpyDeviceToDevice, s));
            for (int l = nl - 1; l >= 1; --l) {
                dalloc(ctx, ctx->L[l - 1].cell_nu, ctx->L[l - 1].nc);
                CK(launch_nu_average(ctx->L[l], ctx->L[l].cell_nu.p, ctx->L[l - 1].cell_nu.p, s));
            }
        }
        // convecting field (Oseen): kept for the load, recovery and adjoint passes
        REQUIRE(!prm->newton_u || prm->conv, "newton_u needs conv (the previous velocity at the lattice)");
        ctx->has_conv = prm->conv != nullptr;
        ctx->conv_t = 0;
        if (ctx->has_conv) {
            const size_t n = (size_t)ctx->L[nl - 1].nc * (prm->k + 2) * (prm->k + 3);
            dalloc(ctx, ctx->conv_k, n);
            CK(cudaMemcpyAsync(ctx->conv_k.p, prm->conv, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        }
        ctx->has_newton = prm->newton_u != nullptr;
        if (ctx->has_newton) {
            const size_t n = (size_t)ctx->L[nl - 1].n_int * 2 * (prm->k + 1);
            dalloc(ctx, ctx->newton_x, std::max<size_t>(n, 1));
            CK(cudaMemcpyAsync(ctx->newton_x.p, prm->newton_u, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        }
        condense_all(ctx, forcing, s);
        // inhomogeneous Dirichlet data: a copy, the cells' boundary fluxes and the load coupling
        ctx->has_dir = prm->dirichlet != nullptr;
        if (ctx->has_dir) {
            DevLevel &F = ctx->L[nl - 1];
            const size_t nb = (size_t)F.n_bnd * 2 * (prm->k + 1);
            dalloc(ctx, ctx->dir_x, std::max<size_t>(nb, 1));
            CK(cudaMemcpyAsync(ctx->dir_x.p, prm->dirichlet, sizeof(double) * nb, cudaMemcpyDeviceToDevice, s));
            dalloc(ctx, ctx->dir_flux, std::max<int64_t>(F.nc, 1));
            CK(launch_boundary_flux(F, 2 * (prm->k + 1), ctx->dir_x.p, ctx->dir_flux.p, s));
        }
        if (rhs_out) {
            if (forcing) CK(launch_assemble_load(ctx->L[nl - 1], ctx->opk, rhs_out, s));
            else CK(cudaMemsetAsync(rhs_out, 0, sizeof(double) * ctx->n_dof, s));
            if (ctx->has_dir) CK(launch_dirichlet_load(ctx->L[nl - 1], ctx->opk, ctx->dir_x.p, rhs_out, s));
        }
    });
}

hdg_status hdg_load(hdg_ctx *ctx, const double *forcing, double *rhs_out, hdg_stream_t stream) {
    if (!ctx) return HDG_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        if (!ctx->condensed) { ctx->err = "hdg_load before hdg_condense"; throw Fail{HDG_ERR_STATE}; }
        REQUIRE(forcing && rhs_out, "null forcing or rhs_out");
        cudaStream_t s = (cudaStream_t)stream;
        load_impl(ctx, forcing, rhs_out, s);
    });
}

#define NEED_2D(what)                                                                        \
    do {                                                                                     \
        if (ctx->dim != 2) {                                                                 \
            ctx->err = std::string(what) + " is available for triangular meshes (dim = 2) only"; \
            throw Fail{HDG_ERR_UNSUPPORTED};                                                 \
        }                                                                                    \
    } while (0)

#define NEED_CONDENSED()                                                                     \
    do {                                                                                     \
        if (!ctx->condensed) {                                                               \
            ctx->err = "operator used before hdg_condense";                                  \
            throw Fail{HDG_ERR_STATE};                                                       \
        }                                                                                    \
    } while (0)

hdg_status hdg_apply(hdg_ctx *ctx, const double *x, double *y, hdg_stream_t stream) {
    if (!ctx) return HDG_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        NEED_CONDENSED();
        REQUIRE(x && y && x != y, "x, y must be distinct non-null device pointers");
        apply_k(ctx, x, nullptr, y, (cudaStream_t)stream);
    });
}

hdg_status hdg_apply_transpose(hdg_ctx *ctx, int level, const double *x, double *y, hdg_stream_t stream) {
    if (!ctx) return HDG_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        NEED_2D("hdg_apply_transpose");
        NEED_CONDENSED();
        REQUIRE(level >= -1 && level < ctx->n_levels, "level out of range");
        REQUIRE(x && y && x != y, "x, y must be distinct non-null device pointers");
        const DevLevel &L = ctx->L[level < 0 ? ctx->n_levels - 1 : level];
        CK(launch_apply_t(L, level < 0 ? ctx->opk : L.op0, x, y, (cudaStream_t)stream));
    });
}

hdg_status hdg_precond_apply(hdg_ctx *ctx, const double *r, double *z, hdg_stream_t stream) {
    if (!ctx) return HDG_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        NEED_CONDENSED();
        REQUIRE(r && z && r != z, "r, z must be distinct non-null device pointers");
        precond(ctx, r, z, (cudaStream_t)stream);
        check_wait_flag_sweep(ctx, (cudaStream_t)stream);
    });
}

hdg_status hdg_level_apply(hdg_ctx *ctx, int level, const double *x, double *y, hdg_stream_t stream) {
    if (!ctx) return HDG_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        NEED_CONDENSED();
        REQUIRE(level >= -1 && level < ctx->n_levels, "level out of range");
        REQUIRE(x && y && x != y, "x, y must be distinct non-null device pointers");
        cudaStream_t s = (cudaStream_t)stream;
        if (level < 0) apply_k(ctx, x, nullptr, y, s);
        else CK(launch_apply<double>(ctx->L[level], ctx->L[level].op0, ctx->L[level].op0.A.p, x, nullptr, y, s));
    });
}

hdg_status hdg_smooth(hdg_ctx *ctx, int level, const double *g, double *u, int n_sweeps, int reverse,
                      hdg_stream_t stream) {
    if (!ctx) return HDG_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        NEED_CONDENSED();
        REQUIRE(level >= -1 && level < ctx->n_levels, "level out of range");
        REQUIRE(g && u && n_sweeps >= 0, "bad arguments");
        cudaStream_t s = (cudaStream_t)stream;
        const int J = ctx->n_levels - 1;
        DevLevel &L = ctx->L[level < 0 ? J : level];
        const DevOperator &op = level < 0 ? ctx->opk : L.op0;
        const int64_t n = L.n_int * op.dpf;
        if (ctx->prm.precision == HDG_FP64) {
            for (int i = 0; i < n_sweeps; ++i) sweep<double>(ctx, L, op, g, u, reverse != 0, s);
        } else {
            float *gf = level < 0 ? ctx->kgf.p : L.gf.p, *uf = level < 0 ? ctx->kuf.p : L.uf.p;
            CK(launch_d2f(g, gf, n, s));
            CK(launch_d2f(u, uf, n, s));
            for (int i = 0; i < n_sweeps; ++i) sweep<float>(ctx, L, op, gf, uf, reverse != 0, s);
            CK(launch_f2d(uf, u, n, s));
            if (level < 0) check_wait_flag_sweep(ctx, s);
        }
    });
}

hdg_status hdg_set_wait_limit(hdg_ctx *ctx, int64_t first_wait_ns) {
    if (!ctx) return HDG_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        REQUIRE(first_wait_ns >= 0, "first_wait_ns must be >= 0");
        ctx->opk.tma_wait_ns = (unsigned long long)first_wait_ns;
        drop_graph(ctx);   // the captured preconditioner holds the old limit
    });
}

hdg_status hdg_prolong_add(hdg_ctx *ctx, int level, const double *uc, double *uf, hdg_stream_t stream) {
    if (!ctx) return HDG_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        NEED_CONDENSED();
        REQUIRE(level >= 1 && level < ctx->n_levels, "level out of range 1..n_levels-1");
        REQUIRE(uc && uf, "null vector");
        DevLevel &F = ctx->L[level];
        CK(launch_prolong_add<double>(F, ctx->L[level - 1], F.tr_W.p, F.tr_H.p, uc, F.t.p, uf,
                                      (cudaStream_t)stream));
    });
}

hdg_status hdg_restrict(hdg_ctx *ctx, int level, const double *rf, double *rc, hdg_stream_t stream) {
    if (!ctx) return HDG_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        NEED_CONDENSED();
        REQUIRE(level >= 1 && level < ctx->n_levels, "level out of range 1..n_levels-1");
        REQUIRE(rf && rc, "null vector");
        DevLevel &F = ctx->L[level];
        CK(launch_restrict<double>(F, ctx->L[level - 1], F.tr_W.p, F.tr_H.p, rf, F.ct1.p, F.ct2.p, rc,
                                   (cudaStream_t)stream));
    });
}

hdg_status hdg_coarse_solve(hdg_ctx *ctx, const double *g, double *u, hdg_stream_t stream) {
    if (!ctx) return HDG_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        NEED_CONDENSED();
        REQUIRE(g && u && g != u, "g, u must be distinct non-null device pointers");
        CK(launch_coarse_apply(ctx->coarse_inv.p, ctx->n0, g, u, (cudaStream_t)stream));
    });
}

hdg_status hdg_mg_h(hdg_ctx *ctx, const double *g, double *u, hdg_stream_t stream) {
    if (!ctx) return HDG_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        NEED_CONDENSED();
        REQUIRE(g && u, "null vector");
        cudaStream_t s = (cudaStream_t)stream;
        const int J = ctx->n_levels - 1;
        DevLevel &L = ctx->L[J];
        const int64_t n = L.dim * L.n_int;
        if (ctx->prm.precision == HDG_FP64) {
            CK(cudaMemcpyAsync(L.g.p, g, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
            mg_h<double>(ctx, J, ctx->prm.m_h, true, s);
            CK(cudaMemcpyAsync(u, L.u.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        } else {
            CK(launch_d2f(g, L.gf.p, n, s));
            mg_h<float>(ctx, J, ctx->prm.m_h, true, s);
            CK(launch_f2d(L.uf.p, u, n, s));
        }
    });
}

hdg_status hdg_get_element_matrices(hdg_ctx *ctx, int level, double *out, hdg_stream_t stream) {
    if (!ctx) return HDG_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        NEED_CONDENSED();
        REQUIRE(level >= -1 && level < ctx->n_levels, "level out of range");
        REQUIRE(out, "null output");
        const DevOperator &op = level < 0 ? ctx->opk : ctx->L[level].op0;
        const int64_t nc = ctx->L[level < 0 ? ctx->n_levels - 1 : level].nc;
        // the library keeps each A_K by row blocks; hand out the row-major A_K[p][q]
        CK(launch_unpack_blocks(nc, op.nloc, op.dpf, op.A.p, out, (cudaStream_t)stream));
    });
}

hdg_status hdg_solve(hdg_ctx *ctx, const double *F, double *u, double *p, const hdg_solve_opts *opts_in,
                     hdg_solve_info *info, hdg_stream_t stream) {
    if (!ctx) return HDG_ERR_INVALID_ARG;
    hdg_solve_info loc{};
    hdg_status conv = HDG_OK;
    hdg_status st = guard(ctx, [&] {
        NEED_CONDENSED();
        REQUIRE(F && u && p, "null vector");
        conv = uzawa_solve(ctx, F, u, p, opts_in, loc, (cudaStream_t)stream);
        check_wait_flag(ctx, (cudaStream_t)stream);
    });
    if (info) *info = loc;
    if (st != HDG_OK) return st;
    if (conv != HDG_OK) ctx->err = "iteration limit reached";
    return conv;
}

hdg_status hdg_recover(hdg_ctx *ctx, const double *u, const double *forcing, double *L_out, double *ulat_out,
                       hdg_stream_t stream) {
    if (!ctx) return HDG_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        NEED_CONDENSED();
        REQUIRE(u, "null skeleton vector");
        cudaStream_t s = (cudaStream_t)stream;
        if (ctx->dim == 3) {
            // the condensation kernel in recovery mode on the finest level (forcing may be NULL)
            DevLevel &LJ = ctx->L[ctx->n_levels - 1];
            int sms = 0;
            CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
            Recover3 rec;
            rec.x = u;
            rec.cell_int = LJ.cell_int.p;
            if (ctx->has_dir) {
                rec.cell_bnd = LJ.cell_bnd.p;
                rec.xD = ctx->dir_x.p;
            }
            rec.L = L_out;
            rec.ulat = ulat_out;
            CK(launch_condense3(ctx->prm.k, LJ, ctx->ref3k_dev.p, ctx->ref3k, ctx->prm.nu, nullptr, ctx->prm.beta,
                                ctx->prm.gamma, forcing, nullptr, nullptr, nullptr, ctx->c3_scratch.p,
                                2 * std::max(sms, 1), ctx->status_flag.p, s, rec));
            check_flag(ctx, s);
            return;
        }
        if (!forcing) {
            const int64_t nlat = (ctx->prm.k + 2) * (ctx->prm.k + 3) / 2;
            dalloc(ctx, ctx->rec_e, (size_t)ctx->L[ctx->n_levels - 1].nc * 2 * nlat);
            CK(cudaMemsetAsync(ctx->rec_e.p, 0, sizeof(double) * ctx->rec_e.n, s));
            forcing = ctx->rec_e.p;
        }
        recover_impl(ctx, u, forcing, L_out, nullptr, ulat_out, s);
    });
}

hdg_status hdg_postprocess(hdg_ctx *ctx, const double *u, const double *forcing, double *ustar_out,
                           hdg_stream_t stream) {
    if (!ctx) return HDG_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        NEED_CONDENSED();
        REQUIRE(u && ustar_out, "null skeleton vector or output");
        cudaStream_t s = (cudaStream_t)stream;
        const int k = ctx->prm.k;
        DevLevel &LJ = ctx->L[ctx->n_levels - 1];
        if (ctx->dim == 3) {
            // recovery (L_h over the orthonormal P^k basis, u_h at the lattice), then u* per cell
            const int64_t nlat = (k + 2) * (k + 3) * (k + 4) / 6, npk = (k + 1) * (k + 2) * (k + 3) / 6;
            if (ctx->post_k != 100 + k || !ctx->post_tabs.p) {
                std::vector<double> t(ctx->ref3k.P1);
                t.insert(t.end(), ctx->ref3k.P2.begin(), ctx->ref3k.P2.end());
                t.insert(t.end(), ctx->ref3k.P3.begin(), ctx->ref3k.P3.end());
                dfree(ctx->post_tabs);
                upload(ctx, ctx->post_tabs, t);
                ctx->post_k = 100 + k;
            }
            dalloc(ctx, ctx->rec_L, (size_t)LJ.nc * 9 * npk);
            dalloc(ctx, ctx->rec_ulat, (size_t)LJ.nc * 3 * nlat);
            int sms = 0;
            CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
            Recover3 rec;
            rec.x = u;
            rec.cell_int = LJ.cell_int.p;
            if (ctx->has_dir) {
                rec.cell_bnd = LJ.cell_bnd.p;
                rec.xD = ctx->dir_x.p;
            }
            rec.L = ctx->rec_L.p;
            rec.ulat = ctx->rec_ulat.p;
            CK(launch_condense3(k, LJ, ctx->ref3k_dev.p, ctx->ref3k, ctx->prm.nu, nullptr, ctx->prm.beta,
                                ctx->prm.gamma, forcing, nullptr, nullptr, nullptr, ctx->c3_scratch.p,
                                2 * std::max(sms, 1), ctx->status_flag.p, s, rec));
            CK(launch_poststar3(k, LJ, ctx->prm.nu, ctx->post_tabs.p, (int)nlat, (int)npk, ctx->rec_L.p,
                                ctx->rec_ulat.p, ustar_out, s));
            check_flag(ctx, s);
            return;
        }
        const int64_t nlat = (k + 2) * (k + 3) / 2, npk = (k + 1) * (k + 2) / 2;
        if (ctx->post_k != k || !ctx->post_tabs.p) {
            std::vector<double> t(ctx->refk.P1);
            t.insert(t.end(), ctx->refk.P2.begin(), ctx->refk.P2.end());
            t.insert(t.end(), ctx->refk.P3.begin(), ctx->refk.P3.end());
            upload(ctx, ctx->post_tabs, t);
            ctx->post_k = k;
        }
        if (!forcing) {
            dalloc(ctx, ctx->rec_e, (size_t)LJ.nc * 2 * nlat);
            CK(cudaMemsetAsync(ctx->rec_e.p, 0, sizeof(double) * ctx->rec_e.n, s));
            forcing = ctx->rec_e.p;
        }
        dalloc(ctx, ctx->rec_L, (size_t)LJ.nc * 4 * npk);
        dalloc(ctx, ctx->rec_ulat, (size_t)LJ.nc * 2 * nlat);
        recover_impl(ctx, u, forcing, ctx->rec_L.p, nullptr, ctx->rec_ulat.p, s);
        CK(launch_poststar(k, LJ, ctx->prm.nu, cell_nu_of(ctx, ctx->n_levels - 1), ctx->post_tabs.p, (int)nlat,
                           (int)npk, ctx->rec_L.p, ctx->rec_ulat.p, ustar_out, s));
    });
}

hdg_status hdg_adjoint(hdg_ctx *ctx, const double *forcing, const double *u, const double *u_target,
                       double *grad_forcing, double *grad_nu, double *J, const hdg_solve_opts *opts,
                       hdg_solve_info *info, hdg_stream_t stream) {
    if (!ctx) return HDG_ERR_INVALID_ARG;
    hdg_solve_info loc{};
    hdg_status conv = HDG_OK;
    hdg_status st = guard(ctx, [&] {
        NEED_2D("hdg_adjoint");
        NEED_CONDENSED();
        REQUIRE(forcing && u && u_target, "null input");
        if (ctx->has_dir) {
            ctx->err = "hdg_adjoint takes homogeneous Dirichlet data only";
            throw Fail{HDG_ERR_UNSUPPORTED};
        }
        if (ctx->has_newton) {
            ctx->err = "hdg_adjoint of a Newton-step operator is not implemented";
            throw Fail{HDG_ERR_UNSUPPORTED};
        }
        cudaStream_t s = (cudaStream_t)stream;
        const int Jl = ctx->n_levels - 1;
        DevLevel &LJ = ctx->L[Jl];
        const int k = ctx->prm.k;
        const int64_t nc = LJ.nc;
        const int64_t npk = (k + 1) * (k + 2) / 2, nrt = (k + 1) * (k + 3), nlat = (k + 2) * (k + 3) / 2;
        dalloc(ctx, ctx->rec_L, nc * 4 * npk);
        dalloc(ctx, ctx->rec_La, nc * 4 * npk);
        dalloc(ctx, ctx->rec_rt, nc * nrt);
        dalloc(ctx, ctx->rec_ulat, nc * 2 * nlat);
        dalloc(ctx, ctx->rec_e, nc * 2 * nlat);
        dalloc(ctx, ctx->rec_j, nc);
        dalloc(ctx, ctx->adj_F, ctx->n_dof);
        dalloc(ctx, ctx->adj_u, ctx->n_dof);
        dalloc(ctx, ctx->adj_p, nc);
        // primal local fields, the objective and the adjoint load u_h - u_target
        recover_impl(ctx, u, forcing, ctx->rec_L.p, nullptr, ctx->rec_ulat.p, s);
        CK(launch_objective(k, LJ, ctx->refk_dev.p, ctx->refk, ctx->rec_ulat.p, u_target, ctx->rec_e.p,
                            ctx->rec_j.p, s));
        hdg_solve_opts o;
        hdg_default_solve_opts(&o);
        if (opts) o = *opts;
        ensure_krylov(ctx, std::max(1, std::min(o.restart, 32)));
        const double Jval = device_sum(ctx, ctx->rec_j.p, nc, s);
        if (J) *J = Jval;
        // Oseen: operators of the transposed convection for the adjoint system
        const bool transposed = ctx->has_conv;
        if (transposed) {
            ctx->conv_t = 1;
            condense_all(ctx, nullptr, s);
        }
        try {
            load_impl(ctx, ctx->rec_e.p, ctx->adj_F.p, s);
            CK(cudaMemsetAsync(ctx->adj_u.p, 0, sizeof(double) * ctx->n_dof, s));
            CK(cudaMemsetAsync(ctx->adj_p.p, 0, sizeof(double) * nc, s));
            conv = uzawa_solve(ctx, ctx->adj_F.p, ctx->adj_u.p, ctx->adj_p.p, &o, loc, s);
            // adjoint local fields, then the contractions
            recover_impl(ctx, ctx->adj_u.p, ctx->rec_e.p, ctx->rec_La.p, ctx->rec_rt.p, nullptr, s);
            CK(launch_adjoint_gradient(k, LJ, ctx->refk_dev.p, ctx->refk, ctx->prm.nu, cell_nu_of(ctx, Jl),
                                       ctx->rec_L.p, ctx->rec_La.p, ctx->rec_rt.p, grad_nu, grad_forcing, s));
        } catch (...) {
            if (transposed) {
                ctx->conv_t = 0;
                ctx->condensed = false;   // the primal operators are gone; hdg_condense again
            }
            throw;
        }
        if (transposed) {
            ctx->conv_t = 0;
            condense_all(ctx, nullptr, s);
        }
        CK(cudaStreamSynchronize(s));
        check_wait_flag(ctx, s);
    });
    if (info) *info = loc;
    if (st != HDG_OK) return st;
    if (conv != HDG_OK) ctx->err = "adjoint solve: iteration limit reached";
    return conv;
}

// ------------------------------------------------------------------ multi-RHS
hdg_status hdg_apply_multi(hdg_ctx *ctx, int nrhs, const double *x, double *y, hdg_stream_t stream) {
    if (!ctx) return HDG_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        NEED_2D("hdg_apply_multi");
        NEED_CONDENSED();
        REQUIRE(nrhs >= 1 && nrhs <= MAX_NRHS, "nrhs out of range 1..64");
        REQUIRE(x && y, "null vector");
        cudaStream_t s = (cudaStream_t)stream;
        const int R = pad_width(nrhs);
        const int64_t n = ctx->n_dof;
        dalloc(ctx, ctx->mrd, (size_t)std::max<int64_t>(n, 1) * R);
        dalloc(ctx, ctx->mzd, (size_t)std::max<int64_t>(n, 1) * R);
        CK(launch_pack_m(x, nrhs, n, R, ctx->mrd.p, s));
        CK(launch_apply_m<double>(ctx->L[ctx->n_levels - 1], ctx->opk, R, ctx->opk.A.p, ctx->mrd.p, nullptr,
                                  ctx->mzd.p, s));
        CK(launch_unpack_m(ctx->mzd.p, nrhs, n, R, y, s));
    });
}

hdg_status hdg_precond_apply_multi(hdg_ctx *ctx, int nrhs, const double *r, double *z, hdg_stream_t stream) {
    if (!ctx) return HDG_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        NEED_2D("hdg_precond_apply_multi");
        NEED_CONDENSED();
        REQUIRE(nrhs >= 1 && nrhs <= MAX_NRHS, "nrhs out of range 1..64");
        REQUIRE(r && z, "null vector");
        cudaStream_t s = (cudaStream_t)stream;
        const int R = pad_width(nrhs);
        const int64_t n = ctx->n_dof;
        dalloc(ctx, ctx->mrd, (size_t)std::max<int64_t>(n, 1) * R);
        dalloc(ctx, ctx->mzd, (size_t)std::max<int64_t>(n, 1) * R);
        CK(launch_pack_m(r, nrhs, n, R, ctx->mrd.p, s));
        precond_m(ctx, ctx->mrd.p, ctx->mzd.p, R, s);
        CK(launch_unpack_m(ctx->mzd.p, nrhs, n, R, z, s));
    });
}

hdg_status hdg_smooth_multi(hdg_ctx *ctx, int level, int nrhs, const double *g, double *u, int n_sweeps,
                            int reverse, hdg_stream_t stream) {
    if (!ctx) return HDG_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        NEED_2D("hdg_smooth_multi");
        NEED_CONDENSED();
        REQUIRE(level >= -1 && level < ctx->n_levels, "level out of range");
        REQUIRE(nrhs >= 1 && nrhs <= MAX_NRHS, "nrhs out of range 1..64");
        REQUIRE(g && u && n_sweeps >= 0, "bad arguments");
        cudaStream_t s = (cudaStream_t)stream;
        const int R = pad_width(nrhs);
        const int J = ctx->n_levels - 1;
        const DevLevel &L = ctx->L[level < 0 ? J : level];
        const DevOperator &op = level < 0 ? ctx->opk : L.op0;
        const int64_t n = L.n_int * op.dpf;
        const size_t nR = (size_t)std::max<int64_t>(n, 1) * R;
        dalloc(ctx, ctx->mrd, nR);
        dalloc(ctx, ctx->mzd, nR);
        CK(launch_pack_m(g, nrhs, n, R, ctx->mrd.p, s));
        CK(launch_pack_m(u, nrhs, n, R, ctx->mzd.p, s));
        if (ctx->prm.precision == HDG_FP64) {
            for (int i = 0; i < n_sweeps; ++i) sweep_m<double>(ctx, L, op, R, ctx->mrd.p, ctx->mzd.p, reverse != 0, s);
        } else {
            dalloc(ctx, ctx->mkgf, nR);
            dalloc(ctx, ctx->mkuf, nR);
            CK((launch_convert_m<double, float>(ctx->mrd.p, ctx->mkgf.p, (int64_t)nR, s)));
            CK((launch_convert_m<double, float>(ctx->mzd.p, ctx->mkuf.p, (int64_t)nR, s)));
            for (int i = 0; i < n_sweeps; ++i)
                sweep_m<float>(ctx, L, op, R, ctx->mkgf.p, ctx->mkuf.p, reverse != 0, s);
            CK((launch_convert_m<float, double>(ctx->mkuf.p, ctx->mzd.p, (int64_t)nR, s)));
        }
        CK(launch_unpack_m(ctx->mzd.p, nrhs, n, R, u, s));
    });
}

hdg_status hdg_set_batched_tile(hdg_ctx *ctx, int rows_per_thread, int threads) {
    if (!ctx) return HDG_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        REQUIRE(rows_per_thread == 0 || rows_per_thread == 1 || rows_per_thread == 2 || rows_per_thread == 4,
                "rows_per_thread must be 0, 1, 2 or 4");
        REQUIRE(threads == 0 || threads == 128 || threads == 256, "threads must be 0, 128 or 256");
        REQUIRE((rows_per_thread == 0) == (threads == 0), "give both or neither");
        REQUIRE(rows_per_thread == 0 || ctx->prm.k == 0 || ctx->opk.dpf % rows_per_thread == 0 || !ctx->condensed,
                "rows_per_thread must divide 2(k+1)");
        ctx->tile_force_rb = rows_per_thread;
        ctx->tile_force_nt = threads;
        drop_graph(ctx);
    });
}

hdg_status hdg_tune_batched(hdg_ctx *ctx, int nrhs, int *rows_per_thread, int *threads, double *ms,
                            hdg_stream_t stream) {
    if (!ctx) return HDG_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        NEED_2D("hdg_tune_batched");
        NEED_CONDENSED();
        REQUIRE(nrhs >= 1 && nrhs <= MAX_NRHS, "nrhs out of range 1..64");
        cudaStream_t s = (cudaStream_t)stream;
        const int R = pad_width(nrhs), li = log2_width(R), pi = ctx->prm.precision == HDG_FP64 ? 0 : 1;
        const int frb = ctx->tile_force_rb, fnt = ctx->tile_force_nt;
        ctx->tile_force_rb = ctx->tile_force_nt = 0;
        const bool tc = pi == 1 && gs_tc_supported(ctx->L[ctx->n_levels - 1], ctx->opk, R);
        ctx->tile_rb[pi][li] = ctx->tile_nt[pi][li] = 0;
        ctx->tile_ms[pi][li] = 0.0;
        ctx->tile_tc_nt[li] = 0;
        ctx->tile_tc_ms[li] = 0.0;
        try {
            ensure_tuned(ctx, R, s);
        } catch (...) {
            ctx->tile_force_rb = frb;
            ctx->tile_force_nt = fnt;
            throw;
        }
        ctx->tile_force_rb = frb;
        ctx->tile_force_nt = fnt;
        drop_graph(ctx);
        // the tensor-core sweep reports 0 rows per thread and its block size
        if (rows_per_thread) *rows_per_thread = tc ? 0 : ctx->tile_rb[pi][li];
        if (threads) *threads = tc ? ctx->tile_tc_nt[li] : ctx->tile_nt[pi][li];
        if (ms) *ms = tc ? ctx->tile_tc_ms[li] : ctx->tile_ms[pi][li];
    });
}

hdg_status hdg_solve_multi(hdg_ctx *ctx, int nrhs, const double *F, double *u, double *p,
                           const hdg_solve_opts *opts, hdg_solve_info *info, hdg_stream_t stream) {
    if (!ctx) return HDG_ERR_INVALID_ARG;
    std::vector<hdg_solve_info> loc;
    hdg_status conv = HDG_OK;
    hdg_status st = guard(ctx, [&] {
        NEED_2D("hdg_solve_multi");
        NEED_CONDENSED();
        REQUIRE(nrhs >= 1 && nrhs <= MAX_NRHS, "nrhs out of range 1..64");
        REQUIRE(F && u && p, "null vector");
        cudaStream_t s = (cudaStream_t)stream;
        const int R = pad_width(nrhs);
        const int64_t n = ctx->n_dof, nc = ctx->L[ctx->n_levels - 1].nc;
        dalloc(ctx, ctx->mF, (size_t)std::max<int64_t>(n, 1) * R);
        dalloc(ctx, ctx->mU, (size_t)std::max<int64_t>(n, 1) * R);
        dalloc(ctx, ctx->mP, (size_t)std::max<int64_t>(nc, 1) * R);
        CK(launch_pack_m(F, nrhs, n, R, ctx->mF.p, s));
        CK(launch_pack_m(u, nrhs, n, R, ctx->mU.p, s));
        CK(launch_pack_m(p, nrhs, nc, R, ctx->mP.p, s));
        conv = uzawa_solve_m(ctx, nrhs, R, ctx->mF.p, ctx->mU.p, ctx->mP.p, opts, loc, s);
        CK(launch_unpack_m(ctx->mU.p, nrhs, n, R, u, s));
        CK(launch_unpack_m(ctx->mP.p, nrhs, nc, R, p, s));
        CK(cudaStreamSynchronize(s));
    });
    if (info)
        for (int r = 0; r < nrhs && r < (int)loc.size(); ++r) info[r] = loc[r];
    if (st != HDG_OK) return st;
    if (conv != HDG_OK) ctx->err = "iteration limit reached";
    return conv;
}

// ------------------------------------------------------------------ several meshes
hdg_status hdg_solve_batched(hdg_ctx *const *ctxs, int n, const double *const *F, double *const *u,
                             double *const *p, const hdg_solve_opts *opts, hdg_solve_info *info,
                             hdg_status *status) {
    if (!ctxs || n < 1 || !F || !u || !p) return HDG_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i]) return HDG_ERR_INVALID_ARG;
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return HDG_ERR_INVALID_ARG;   // one thread per context
    }
    // the calling thread runs context 0 and switches devices: its current device is restored
    int caller_dev = -1;
    if (cudaGetDevice(&caller_dev) != cudaSuccess) return HDG_ERR_CUDA;
    struct RestoreDevice {
        int d;
        ~RestoreDevice() { cudaSetDevice(d); }
    } restore{caller_dev};
    std::vector<hdg_status> st(n, HDG_OK);
    std::vector<hdg_solve_info> inf(n);
    for (int i = 0; i < n; ++i) {
        hdg_ctx *ctx = ctxs[i];
        if (!ctx->batch_stream) {
            cudaSetDevice(ctx->device);
            if (cudaStreamCreateWithFlags(&ctx->batch_stream, cudaStreamNonBlocking) != cudaSuccess) {
                ctx->batch_stream = nullptr;
                ctx->err = "stream creation failed";
                return HDG_ERR_CUDA;
            }
        }
    }
    auto work = [&](int i) {
        hdg_ctx *ctx = ctxs[i];
        if (cudaSetDevice(ctx->device) != cudaSuccess) {
            st[i] = HDG_ERR_CUDA;
            return;
        }
        st[i] = hdg_solve(ctx, F[i], u[i], p[i], opts, &inf[i], (hdg_stream_t)ctx->batch_stream);
    };
    std::vector<std::thread> th;
    th.reserve(n);
    try {
        for (int i = 1; i < n; ++i) th.emplace_back(work, i);
    } catch (...) {
        for (auto &t : th) t.join();
        return HDG_ERR_OOM;
    }
    work(0);
    for (auto &t : th) t.join();
    hdg_status first = HDG_OK;
    for (int i = 0; i < n; ++i) {
        if (info) info[i] = inf[i];
        if (status) status[i] = st[i];
        if (first == HDG_OK && st[i] != HDG_OK) first = st[i];
    }
    return first;
}

// ------------------------------------------------------------------ steady Navier-Stokes (Picard)
hdg_status hdg_picard(hdg_ctx *ctx, const hdg_params *params, const double *forcing, double tol, int max_steps,
                      double *u, double *p, const hdg_solve_opts *opts, int *steps_out, double *dist_out,
                      hdg_stream_t stream) {
    if (!ctx) return HDG_ERR_INVALID_ARG;
    hdg_status conv = HDG_OK;
    int steps = 0;
    double dist = 0.0;
    hdg_status st = guard(ctx, [&] {
        NEED_2D("hdg_picard");
        REQUIRE(params && forcing && u && p, "null argument");
        if (params->dirichlet) {
            ctx->err = "hdg_picard takes homogeneous Dirichlet data only";
            throw Fail{HDG_ERR_UNSUPPORTED};
        }
        REQUIRE(max_steps >= 1 && tol >= 0 && std::isfinite(tol), "bad tol or max_steps");
        REQUIRE(params->k >= 0 && params->k <= MAX_K, "k out of range 0..4");
        REQUIRE(params->pseudo_dt_inv >= 0 && std::isfinite(params->pseudo_dt_inv), "pseudo_dt_inv must be >= 0");
        cudaStream_t s = (cudaStream_t)stream;
        const int J = ctx->n_levels - 1;
        DevLevel &LJ = ctx->L[J];
        const int k = params->k;
        const int64_t nc = LJ.nc, nlat = (k + 2) * (k + 3) / 2, n_dof = LJ.n_int * 2 * (k + 1);
        dalloc(ctx, ctx->pic_F, std::max<int64_t>(n_dof, 1));
        dalloc(ctx, ctx->pic_w0, nc * 2 * nlat);
        dalloc(ctx, ctx->pic_w1, nc * 2 * nlat);
        dalloc(ctx, ctx->pic_e, nc * 2 * nlat);
        dalloc(ctx, ctx->pic_j, std::max<int64_t>(nc, 1));
        auto check = [&](hdg_status r) {
            if (r == HDG_ERR_NOT_CONVERGED) conv = r;
            else if (r != HDG_OK) throw Fail{r};
        };
        // u^(0): the generalized Stokes problem with the same data
        hdg_params prm = *params;
        prm.conv = nullptr;
        prm.newton_u = nullptr;
        check(hdg_condense(ctx, &prm, forcing, ctx->pic_F.p, stream));
        CK(cudaMemsetAsync(u, 0, sizeof(double) * n_dof, s));
        CK(cudaMemsetAsync(p, 0, sizeof(double) * nc, s));
        check(hdg_solve(ctx, ctx->pic_F.p, u, p, opts, nullptr, stream));
        double *wp = ctx->pic_w0.p, *wc = ctx->pic_w1.p;
        recover_impl(ctx, u, forcing, nullptr, nullptr, wp, s);
        // Oseen steps with w_h = u_h^(n-1) until ||u^(n) - u^(n-1)|| < tol; with pseudo-time the
        // step adds (u^n - u^(n-1))/dt*: beta + 1/dt* and the load f + u^(n-1)/dt*
        const double dti = params->pseudo_dt_inv;
        prm.beta = params->beta + dti;
        if (dti > 0) dalloc(ctx, ctx->pic_f, nc * 2 * nlat);
        for (int n = 1; n <= max_steps; ++n) {
            prm.conv = wp;
            const double *fn = forcing;
            if (dti > 0) {
                CK(cudaMemcpyAsync(ctx->pic_f.p, forcing, sizeof(double) * nc * 2 * nlat, cudaMemcpyDeviceToDevice, s));
                CK(launch_axpby(dti, wp, 1.0, ctx->pic_f.p, nc * 2 * nlat, s));
                fn = ctx->pic_f.p;
            }
            check(hdg_condense(ctx, &prm, fn, ctx->pic_F.p, stream));
            check(hdg_solve(ctx, ctx->pic_F.p, u, p, opts, nullptr, stream));
            recover_impl(ctx, u, fn, nullptr, nullptr, wc, s);
            CK(launch_objective(k, LJ, ctx->refk_dev.p, ctx->refk, wc, wp, ctx->pic_e.p, ctx->pic_j.p, s));
            dist = std::sqrt(std::max(2.0 * device_sum(ctx, ctx->pic_j.p, nc, s), 0.0));
            steps = n;
            std::swap(wp, wc);
            if (!std::isfinite(dist)) {
                ctx->err = "non-finite Picard update";
                throw Fail{HDG_ERR_NONFINITE};
            }
            if (dist < tol) break;
        }
        if (!(dist < tol) && conv == HDG_OK) conv = HDG_ERR_NOT_CONVERGED;
        CK(cudaStreamSynchronize(s));
        check_wait_flag(ctx, s);
    });
    if (steps_out) *steps_out = steps;
    if (dist_out) *dist_out = dist;
    if (st != HDG_OK) return st;
    if (conv != HDG_OK) ctx->err = "Picard iteration or an inner solve reached its limit";
    return conv;
}

hdg_status hdg_newton(hdg_ctx *ctx, const hdg_params *params, const double *forcing, double tol, int max_steps,
                      double *u, double *p, const hdg_solve_opts *opts, int *steps_out, double *dist_out,
                      hdg_stream_t stream) {
    if (!ctx) return HDG_ERR_INVALID_ARG;
    hdg_status conv = HDG_OK;
    int steps = 0;
    double dist = 0.0;
    hdg_status st = guard(ctx, [&] {
        NEED_2D("hdg_newton");
        NEED_CONDENSED();
        REQUIRE(params && forcing && u && p, "null argument");
        if (params->dirichlet || ctx->has_dir) {
            ctx->err = "hdg_newton takes homogeneous Dirichlet data only";
            throw Fail{HDG_ERR_UNSUPPORTED};
        }
        REQUIRE(max_steps >= 1 && tol >= 0 && std::isfinite(tol), "bad tol or max_steps");
        REQUIRE(params->k == ctx->prm.k, "params->k differs from the condensed operator's k");
        cudaStream_t s = (cudaStream_t)stream;
        DevLevel &LJ = ctx->L[ctx->n_levels - 1];
        const int k = params->k;
        const int64_t nc = LJ.nc, nlat = (k + 2) * (k + 3) / 2, n_dof = ctx->n_dof;
        dalloc(ctx, ctx->pic_F, std::max<int64_t>(n_dof, 1));
        dalloc(ctx, ctx->pic_w0, nc * 2 * nlat);
        dalloc(ctx, ctx->pic_w1, nc * 2 * nlat);
        dalloc(ctx, ctx->pic_e, nc * 2 * nlat);
        dalloc(ctx, ctx->pic_j, std::max<int64_t>(nc, 1));
        dalloc(ctx, ctx->pic_x, std::max<int64_t>(n_dof, 1));   // previous skeleton iterate
        auto check = [&](hdg_status r) {
            if (r == HDG_ERR_NOT_CONVERGED) conv = r;
            else if (r != HDG_OK) throw Fail{r};
        };
        double *wp = ctx->pic_w0.p, *wc = ctx->pic_w1.p;
        // the iterate (u, p) was computed with the operator the context holds: recover it with that
        recover_impl(ctx, u, forcing, nullptr, nullptr, wp, s);
        hdg_params prm = *params;
        for (int n = 1; n <= max_steps; ++n) {
            CK(cudaMemcpyAsync(ctx->pic_x.p, u, sizeof(double) * n_dof, cudaMemcpyDeviceToDevice, s));
            prm.conv = wp;
            prm.newton_u = ctx->pic_x.p;
            check(hdg_condense(ctx, &prm, forcing, ctx->pic_F.p, stream));
            check(hdg_solve(ctx, ctx->pic_F.p, u, p, opts, nullptr, stream));
            recover_impl(ctx, u, forcing, nullptr, nullptr, wc, s);
            CK(launch_objective(k, LJ, ctx->refk_dev.p, ctx->refk, wc, wp, ctx->pic_e.p, ctx->pic_j.p, s));
            dist = std::sqrt(std::max(2.0 * device_sum(ctx, ctx->pic_j.p, nc, s), 0.0));
            steps = n;
            std::swap(wp, wc);
            if (!std::isfinite(dist)) {
                ctx->err = "non-finite Newton update";
                throw Fail{HDG_ERR_NONFINITE};
            }
            if (dist < tol) break;
        }
        if (!(dist < tol) && conv == HDG_OK) conv = HDG_ERR_NOT_CONVERGED;
        CK(cudaStreamSynchronize(s));
        check_wait_flag(ctx, s);
    });
    if (steps_out) *steps_out = steps;
    if (dist_out) *dist_out = dist;
    if (st != HDG_OK) return st;
    if (conv != HDG_OK) ctx->err = "Newton iteration or an inner solve reached its limit";
    return conv;
}

} // extern "C"
