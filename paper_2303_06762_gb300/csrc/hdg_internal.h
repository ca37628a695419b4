// Internal declarations of the GB300 H(div)-HDG hp-multigrid library.
//
// Host side: topology (facets, orientation, patches, colouring, transfer
// maps) and reference-element tables, built once per mesh hierarchy.
// Device side: condensed element matrices, patch inverses, transfer blocks
// and all hot-path kernels.  See include/hdg.h for the public layouts.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "hdg.h"

namespace hdg {

constexpr int MAX_K = 4;
constexpr int MAX_LEVELS = 16;
constexpr int MAX_RESTART = 64;
constexpr int64_t MAX_COARSE_DOFS = 16384;   // dense inverse of the coarsest level: <= 2 GB

// ---------------------------------------------------------------- host data
struct HostLevel {
    int64_t nv = 0, nc = 0;
    std::vector<double> coords;          // nv*2
    std::vector<int32_t> cells;          // nc*3
    std::vector<int32_t> parent;         // nc (level > 0)
    std::vector<int32_t> colour;         // nv
    // facets
    int64_t nf = 0, n_int = 0;
    std::vector<int32_t> facet_v;        // nf*2 sorted vertex pair
    std::vector<int32_t> cell_facet;     // nc*3 facet opposite local vertex f
    std::vector<int32_t> facet_cells;    // nf*2 (second = -1 on boundary)
    std::vector<int32_t> facet_lf;       // nf*2 local facet index in each cell
    std::vector<int32_t> interior_index; // nf -> interior number or -1
    std::vector<int32_t> interior_facets;// n_int
    // vertex patches, sorted by (colour, vertex id); only non-empty patches
    int n_patches = 0, n_colours = 0, pf_max = 0, pc_max = 0;
    std::vector<int32_t> colour_ptr;     // n_colours+1 offsets into patch order
    std::vector<int32_t> patch_nf;       // n_patches
    std::vector<int32_t> patch_facets;   // n_patches*pf_max interior facet ids (-1 pad)
    std::vector<int32_t> patch_nc;       // n_patches
    std::vector<int32_t> patch_cells;    // n_patches*pc_max
    // for slot j of patch p: the two (star-cell index << 2 | local facet) pairs
    std::vector<int32_t> patch_slot_src; // n_patches*pf_max*2
    // n_patches*pc_max: the local facet of each star cell opposite the patch vertex (-1 pad),
    // the one facet of the cell outside the patch
    std::vector<int32_t> patch_cext;
};

// transfer data between level l-1 (coarse) and l (fine), stored on level l
struct HostTransfer {
    int64_t nc_coarse = 0;
    std::vector<int32_t> slots;      // nc_coarse*9: fine interior facet id per slot or -1
    std::vector<int32_t> nbr;        // nc_coarse*6: (other coarse cell << 4 | its slot) or -1
    std::vector<int32_t> children;   // nc_coarse*4
    std::vector<int32_t> child_slot; // nc_coarse*4*3: slot of each child's local facet
    std::vector<double> W;           // nc_coarse*12*6 averaging weights (eq. avgOpt)
    int64_t nB = 0;
    std::vector<int32_t> fineB;      // nB: fine interior facet id of each B facet
    std::vector<int32_t> fineB_src;  // nB*2: (coarse cell << 4 | slot)
};

// reference-element tables for order k (FP64), see reference.cpp
struct RefTables {
    int k = -1, npk = 0, nrt = 0, nf = 0, nlat = 0, nq = 0, nfq = 0;
    std::vector<double> R1, R2, R3, R4, R5, R6, R7, R8;
    // point values for the upwind convection (reference.cpp)
    std::vector<double> R9, R10, R11, R12, R13, R14, R15, R16;
    // post-processing of eq. stPost (u* in [P^{k+1}]^2, Lagrange basis lam_n of the lattice):
    // P1[(a*2+b)][n][n'] = ∫ d_a lam_n d_b lam_n', P2[j][n][b] = ∫ g_j d_b lam_n, P3[n] = ∫ lam_n
    std::vector<double> P1, P2, P3;
};
constexpr int N_REF_TABLES = 16;

// layout of the small Krylov block (restart R):
//   H: (R+1) x R column-major at 0; cs, sn: R; g: R+1; y: R; h1, h2: R+1; nrm2, res, hn
struct SmallLayout {
    int R;
    __host__ __device__ int H() const { return 0; }
    __host__ __device__ int cs() const { return (R + 1) * R; }
    __host__ __device__ int sn() const { return cs() + R; }
    __host__ __device__ int g() const { return sn() + R; }
    __host__ __device__ int y() const { return g() + R + 1; }
    __host__ __device__ int h1() const { return y() + R; }
    __host__ __device__ int h2() const { return h1() + R + 1; }
    __host__ __device__ int nrm2() const { return h2() + R + 1; }
    __host__ __device__ int res() const { return nrm2() + 1; }
    __host__ __device__ int hn() const { return res() + 1; }
    __host__ __device__ int total() const { return hn() + 1; }
};


// views of the smallest lowest-order levels for the single-block MG kernel (mg_small.cu)
constexpr int SMALL_MAX_LEVELS = 6;
constexpr int64_t GS0_TABLE_MAX_CELLS = int64_t(1) << 25;   // every level up to 33.5M cells (int32 offsets c*36)
constexpr int GS0_TABLE_INTS = 12;
constexpr int SMALL_MAX_COLOURS = 15;
constexpr int64_t SMALL_MAX_CELLS = 32768;

template <class T>
struct SmallLevel {
    int n_int = 0, n_colours = 0, pf_max = 0, pc_max = 0, np_max = 0;
    int colour_ptr[SMALL_MAX_COLOURS + 1] = {};
    const int *cell_int = nullptr, *facet_adj = nullptr, *patch_nf = nullptr, *patch_facets = nullptr,
              *patch_cells = nullptr, *slot_src = nullptr;
    const T *A = nullptr, *Pinv = nullptr;
    T *g = nullptr, *u = nullptr, *r = nullptr, *t = nullptr;
    int ncc = 0, nB = 0;
    const int *tr_slots = nullptr, *tr_nbr = nullptr, *tr_fineB = nullptr, *tr_fineB_src = nullptr;
    const T *W = nullptr, *H = nullptr;
    T *ct1 = nullptr, *ct2 = nullptr;
};

template <class T>
struct SmallParams {
    SmallLevel<T> lv[SMALL_MAX_LEVELS];
    const double *inv = nullptr;   // dense inverse of the coarsest operator (FP64)
    double *g0d = nullptr;         // FP64 staging of the coarsest right-hand side
    int q = 1, growth = 2;
    // single-block launch only: keep every level vector (g, u, r, t, transfer temporaries,
    // the FP64 coarse right-hand side) in shared memory from byte vec_offset on
    int resident = 0;
    size_t vec_offset = 0;
};

// outputs of the recovery mode of the condensation kernel (all device, nullable)
struct RecoverArgs {
    const double *x = nullptr;      // skeleton solution [n_int][dpf]; null = no recovery
    const int *cell_int = nullptr;  // cell -> interior facet
    double *L = nullptr;            // [nc][4*npk] flux coefficients (orthonormal P^k, per component)
    double *rt = nullptr;           // [nc][nrt] RT coefficients in the reference dual basis
    double *po = nullptr;           // [nc][npk-1] mean-free pressure coefficients
    double *ulat = nullptr;         // [nc][nlat][2] velocity at the degree-(k+1) lattice
    const int *cell_bnd = nullptr;  // with xD: boundary facet of each local facet or -1
    const double *xD = nullptr;     // inhomogeneous Dirichlet data [n_boundary][dpf], or null
};

// ---------------------------------------------------------------- device data
template <class T>
struct DBuf {
    T *p = nullptr;
    size_t n = 0;
};

struct DevOperator {
    int k = -1, dpf = 0, nloc = 0, np_max = 0;
    DBuf<double> A;      // nc*nloc*nloc
    DBuf<float> Af;
    DBuf<float> Alo;     // A - (double)Af, for the double-FP32 apply of the batched solver
    bool alo_valid = false;
    DBuf<double> Fel;    // nc*nloc element loads
    DBuf<double> Pinv;   // n_patches*np_max*np_max
    DBuf<float> Pinvf;
    DBuf<float> Pinvp;   // symmetric operators, order k: packed upper triangles of (Pinv + Pinv^T)/2,
                         // packed_patch_size(np_max) floats per patch (bulk-copy sweep)
    // the FP32 closed-form sweep's split of the augmented-Lagrangian term G_c d_c d_c^T
    // (G_c = gamma nu_c / |K|, d_c the cell's flux weights on each facet's first unknown), so that
    // no O(gamma) value meets the FP32 inverse (2D levels with patch_cext, FP32 preconditioners):
    DBuf<float> swQ;     // n_patches*pc_max*np_max: column si of patch p, Q = A_PP^-1 D_P G (np_max
                         // rows at (p pc_max + si) np_max), D_P G the AL columns of the star cells
    DBuf<float> swA00;   // n_patches*pf_max*2: entry (0, 0) of each slot's coupling block with the
                         // cell's outside facet, without the AL term
    // 16-bit copies for HDG_MIXED_BF16 / HDG_MIXED_FP16 (order-k operator only): the
    // layouts of A and Pinv with every stored row divided by its power-of-two scale
    int *tma_flag = nullptr; // device flag of the bulk-copy sweep's bounded waits (bit 4 on timeout),
                             // null = that sweep is not used
    unsigned long long tma_wait_ns = 1000000000ull;   // limit of that sweep's first wait (0 = expire at once)
    int h_fmt = 0;       // hdg_precision of Ah / Pinvh, 0 = none
    DBuf<uint16_t> Ah;   // nc*nloc*nloc
    DBuf<float> Ah_s;    // nc*nloc, scale of row p of cell c at c*nloc + p
    DBuf<uint16_t> Pinvh;
    DBuf<float> Pinvh_s; // n_patches*np_max, scale of row i of the inverse of patch p at p*np_max + i
};

// ---------------------------------------------------------------- 3D host data
constexpr int MAX_K3 = 3;
constexpr int TR3_B = 16;      // fine faces on the faces of a coarse cell (4 per coarse face)
constexpr int TR3_T = 8;       // fine faces inside a coarse cell
constexpr int TR3_SLOTS = TR3_B + TR3_T;

inline int dpf3(int k) { return 3 * (k + 1) * (k + 2) / 2; }
inline int nface3(int k) { return (k + 1) * (k + 2) / 2; }
// skeleton unknowns per facet of an order-k space in dimension dim
inline int dpf_of(int dim, int k) { return dim == 3 ? dpf3(k) : 2 * (k + 1); }

struct HostLevel3 {
    int64_t nv = 0, nc = 0;
    std::vector<double> coords;          // nv*3
    std::vector<int32_t> cells;          // nc*4
    std::vector<int32_t> parent;         // nc (level > 0)
    int64_t nf = 0, n_int = 0;
    std::vector<int32_t> face_v;         // nf*3 sorted vertex triple
    std::vector<int32_t> cell_face;      // nc*4 face opposite local vertex f
    std::vector<int32_t> face_cells;     // nf*2 (second = -1 on the boundary)
    std::vector<int32_t> face_lf;        // nf*2 local face in each cell
    std::vector<int32_t> interior_index; // nf -> interior number or -1
    std::vector<int32_t> interior_faces; // n_int
    int64_t ne = 0;
    std::vector<int32_t> edge_v;         // ne*2 sorted vertex pair
    std::vector<int32_t> colour;         // ne greedy colouring (edges of one colour share no cell)
    // edge patches sorted by (colour, edge id); only edges with an interior face
    int n_patches = 0, n_colours = 0, pf_max = 0, pc_max = 0;
    std::vector<int32_t> colour_ptr, patch_nf, patch_facets, patch_nc, patch_cells, patch_slot_src;
    // n_patches*pc_max*2: the two local faces of each star cell that do not contain the patch
    // edge (the faces opposite its end points; -1 pad)
    std::vector<int32_t> patch_cext;
};

// transfer data between a coarse and its red-refined fine level, stored per coarse cell P:
//   slots[P][s]  fine interior face of slot s: s = 4 cf + i (i < 4) are the fine faces on coarse
//                face cf (B slots), s = 16 + t the faces inside P (T slots); -1 for boundary faces
//   nbr[P][s]    for B slots: (other coarse cell Q << 5 | its slot) or -1
//   child_slot[P][ch][lf]  slot of local face lf of the ch-th child, -1 on the boundary
//   W[P][s][a][j]  averaging weights (eq. avgOpt, the 1/2 of the two sides included): fine
//                unknown a of B slot s from coarse unknown j = 3 cf + a' of P
struct HostTransfer3 {
    int64_t nc_coarse = 0;
    std::vector<int32_t> slots, nbr, children, child_slot;
    std::vector<double> W;
    int64_t nB = 0;
    std::vector<int32_t> fineB, fineB_src;   // per fine face on a coarse interior face: id, 2 x (P << 5 | s)
};

struct RefTables3 {
    int k = -1, npk = 0, nrt = 0, nf = 0, nlat = 0;
    std::vector<double> R1, R2, R3, R4, R5, R6, Q, FA, R7;   // R7: phi at the lattice (recovery)
    // post-processing u* (eq. stPost): P1[(a*3+b)][n][n'] = ∫ d_a lam_n d_b lam_n', P2[j][n][b] = ∫ g_j d_b lam_n,
    // P3[n] = ∫ lam_n (lam_n the Lagrange basis of P^{k+1} on the lattice)
    std::vector<double> P1, P2, P3;
};

struct DevLevel {
    int dim = 2;               // 2: triangles (3 facets per cell, 2 lowest-order unknowns per facet);
                               // 3: tetrahedra (4 faces, 3 unknowns per face, edge patches)
    int64_t nv = 0, nc = 0, n_int = 0;
    DBuf<double> coords;       // nv*2
    DBuf<int32_t> cells;       // nc*3
    DBuf<int32_t> cell_int;    // nc*3 interior facet id or -1
    DBuf<int32_t> facet_adj;   // n_int*2 (cell << 2 | lf) or -1
    DBuf<double> cell_d;       // nc*3 flux weights sigma*sqrt|F| of each local facet
    DBuf<double> cell_nu;      // nc per-cell viscosity (when the caller gives one)
    DBuf<double> cell_area;    // nc
    DBuf<double> conv_flux;    // nc*3 outward fluxes of the convecting field (Oseen)
    DBuf<double> conv_lat;     // nc*3*2 lowest-order convecting field at the vertices
    // patches
    int n_patches = 0, n_colours = 0, pf_max = 0, pc_max = 0;
    std::vector<int32_t> colour_ptr;
    DBuf<int32_t> patch_nf, patch_facets, patch_nc, patch_cells, patch_slot_src;
    DBuf<int32_t> facet_slot;  // n_int*2: the two patch slots (p pf_max + position) holding each facet
    DBuf<int32_t> patch_cint;  // finest level: n_patches*pc_max*3 interior facet of each star cell's local
                               // facets (-1 on the boundary or for padding): the order-k sweep's gather
    DBuf<int32_t> patch_cext;  // the star cells' local facets outside the patch (HostLevel::patch_cext,
                               // HostLevel3::patch_cext): on the finest level in 2D, on every level in 3D
    DBuf<int32_t> cell_bnd;    // nc*3: boundary facet number of each local facet or -1 (finest level)
    int64_t n_bnd = 0;         // boundary facets (finest level)
    // lowest-order sweep gather table (levels with at most GS0_TABLE_MAX_CELLS cells): per
    // patch row t < np_max, GS0_TABLE_INTS ints {row 2F+d, element-row offsets of the two
    // cells c*36 + lf*12 + d, their interior facets (3 each, -1 on the boundary)}; rows
    // t >= np carry row = -1
    DBuf<int32_t> gs0_table;
    DevOperator op0;           // lowest-order condensed operator of this level
    // transfer from level-1
    int64_t nc_coarse = 0, nB = 0;
    DBuf<int32_t> tr_slots, tr_nbr, tr_children, tr_child_slot, tr_fineB, tr_fineB_src;
    DBuf<double> tr_W, tr_H;
    DBuf<float> tr_Wf, tr_Hf;
    // MG work vectors (FP64 and FP32 variants), 2 per interior facet
    DBuf<double> g, u, r, t;
    DBuf<float> gf, uf, rf, tf;
    DBuf<double> ct1, ct2;     // coarse-cell temps for restriction (nc_coarse*12, *6)
    DBuf<float> ct1f, ct2f;
    // multi-right-hand-side MG work (R columns), FP64 and FP32
    DBuf<double> mg, mu, mr, mt, mc1, mc2;
    DBuf<float> mgf, muf, mrf, mtf, mc1f, mc2f;
};

} // namespace hdg

struct hdg_ctx {
    int device = 0;
    int dim = 2;                             // 3: tetrahedral hierarchy (hdg3d paths)
    std::vector<hdg::HostLevel3> H3;
    std::vector<hdg::HostTransfer3> T3;
    hdg::RefTables3 ref3k, ref30;
    hdg::DBuf<double> ref3k_dev, ref30_dev;  // packed 3D reference tables (order k, order 0)
    hdg::DBuf<double> c3_scratch;            // 3D condensation workspace
    std::string err;
    int n_levels = 0;
    std::vector<hdg::HostLevel> H;
    std::vector<hdg::HostTransfer> T;   // T[l] for l >= 1
    std::vector<hdg::DevLevel> L;
    bool condensed = false;
    hdg_params prm{};
    bool has_conv = false;                   // Oseen: convecting field given
    int conv_t = 0;                          // operators built from the transposed convection
    hdg::DBuf<double> conv_k;                // finest convecting field, lattice layout (copy)
    bool has_dir = false;                    // inhomogeneous Dirichlet data given (finest level)
    hdg::DBuf<double> dir_x;                 // its skeleton values [n_boundary][dpf] (copy)
    hdg::DBuf<double> dir_flux;              // per-cell boundary fluxes of the data
    bool has_newton = false;                 // Newton step: previous skeleton iterate below
    hdg::DBuf<double> newton_x;
    hdg::RefTables refk, ref0;
    hdg::DBuf<double> refk_dev, ref0_dev;   // packed R1..R6
    hdg::DevOperator opk;                    // order-k operator on the finest mesh
    int64_t n_dof = 0;
    // order-k vectors (finest)
    hdg::DBuf<double> kr, ku, kt;            // FP64 residual/solution/temp
    hdg::DBuf<float> krf, kuf, kgf;          // FP32 copies
    // coarsest dense inverse
    int64_t n0 = 0;
    hdg::DBuf<double> coarse_inv;
    hdg::DBuf<int> status_flag;              // device error flag
    hdg::DBuf<int> wait_flag;                // set by a kernel whose bounded wait gave up
    // Krylov workspace
    int restart_alloc = 0;
    hdg::DBuf<double> V, Z, w, partials, small;   // small: Hessenberg, rotations, g, y
    hdg::DBuf<double> uz_partials;
    hdg::DBuf<double> jD;                    // damped block Jacobi: patch corrections (FP64 sweeps)
    hdg::DBuf<float> jDf;                    // the same for FP32 sweeps
    hdg::DBuf<double> pcg_buf;               // PCG vectors r, z, p, q (4 n_dof)
    hdg::DBuf<double> post_tabs;             // P1, P2, P3 of the order-k tables (post-processing)
    int post_k = -1;
    double *h_pinned = nullptr;              // host pinned scalars
    double *h_multi = nullptr;               // host pinned per-column scalars (multi-RHS)
    // CUDA graph of one preconditioner application (fixed staging buffers)
    cudaGraphExec_t pc_exec = nullptr;
    cudaStream_t cap_stream = nullptr;       // private stream used only for graph capture
    int pc_prec = -1;
    long long pc_kernels = 0;
    hdg::DBuf<double> pc_in, pc_out;
    // recovery / adjoint workspaces
    hdg::DBuf<double> rec_L, rec_La, rec_rt, rec_ulat, rec_e, rec_j, adj_F, adj_u, adj_p;
    // multi-right-hand-side solves (width mR, restart mRst)
    int mR = 0, mRst = 0;
    hdg::DBuf<double> mV, mZ, mw, mpart, msmall, mhbuf, mF, mU, mP, mG, mkr, mkt, mrd, mzd;
    hdg::DBuf<float> mkgf, mkuf, mkrf;
    hdg::DBuf<float2> mxs;                    // (hi, lo) split of the outer operator's input
    hdg::DBuf<int> mint;                      // per-column ints (m_r, frozen flags)
    cudaGraphExec_t pcm_exec = nullptr;      // graph of one multi preconditioner application
    int pcm_prec = -1, pcm_R = 0;
    // tile of the batched order-k sweep on CUDA cores (rows per thread, threads per block):
    // forced by hdg_set_batched_tile, else chosen by the autotuner per (FP64 or FP32, log2 R)
    int tile_force_rb = 0, tile_force_nt = 0;
    int tile_rb[2][7] = {}, tile_nt[2][7] = {};
    double tile_ms[2][7] = {};
    int tile_tc_nt[7] = {};                  // tensor-core sweep: threads per block per log2 R (autotuned)
    double tile_tc_ms[7] = {};
    hdg::DBuf<double> tune_buf;
    long long pcm_kernels = 0;
    hdg::DBuf<double> pcm_in, pcm_out;
    cudaStream_t batch_stream = nullptr;     // private stream for hdg_solve_batched
    hdg::DBuf<double> pic_F, pic_w0, pic_w1, pic_e, pic_j, pic_x;   // Picard / Newton iteration work
    hdg::DBuf<double> pic_f;                 // Picard with pseudo-time: the step's lattice load
    // fused MG_h on levels 0..small_Ls (one thread block), -1 when not used
    int small_Ls = -1;
    size_t small_smem_d = 0, small_smem_f = 0;   // per-CTA shared memory of the fused kernel
    int small_cs_d = 1, small_cs_f = 1;          // its cluster size
    hdg::SmallParams<double> small_d;
    hdg::SmallParams<float> small_f;
};

namespace hdg {

// floats of one packed symmetric patch inverse: np(np+1)/2 rounded up to 4 (16 bytes)
inline int packed_patch_size(int np_max) { return (np_max * (np_max + 1) / 2 + 3) / 4 * 4; }

// kernel-launch counter (ops.cu): every launcher adds the kernels it enqueues
void note_launches(long long n);
unsigned long long launch_count();
unsigned long long thread_launch_count();   // this host thread's share (graph capture bookkeeping)

// reference.cpp
void build_reference_tables(int k, RefTables &out);
size_t ref_table_offset(const RefTables &t, int which);   // offset of R1..R16 in packed buffer
const std::vector<double> *ref_table(const RefTables &t, int which);   // R(which+1)

// topology.cpp
std::string build_level_topology(HostLevel &L, const int32_t *colour_or_null);
std::string build_transfer(const HostLevel &coarse, const HostLevel &fine, HostTransfer &T);

// kernels: condensation and setup (condense.cu)
// conv: lattice values of the convecting field (NULL = Stokes); conv_t: use the
// transposed convection block (adjoint system)
// newton_x: previous skeleton iterate [n_int][dpf] for the Newton term (requires conv), or NULL
cudaError_t launch_condense(int k, const DevLevel &L, const double *ref, const RefTables &rt,
                            double nu, const double *nu_cell, double beta, double gamma,
                            const double *forcing, const double *conv, int conv_t, const double *newton_x,
                            double *A, float *Af, double *Fel, int *flag, const RecoverArgs &rec, cudaStream_t s);
cudaError_t launch_conv_flux(const DevLevel &L, const double *ref, const RefTables &rt, const double *conv,
                             double *flux, cudaStream_t s);
cudaError_t launch_flux_restrict(const DevLevel &fine, const double *ff, double *fc, cudaStream_t s);
cudaError_t launch_rt0_vertex(const DevLevel &L, const double *flux, double *out, cudaStream_t s);
cudaError_t launch_unpack_blocks(int64_t nblk, int n, int dpf, const double *in, double *out, cudaStream_t s);
// pivot: partial pivoting (non-symmetric patch matrices); without it SPD pivots are checked positive
cudaError_t launch_patch_inverse(const DevLevel &L, const DevOperator &op, int pivot, int *flag, cudaStream_t s);
cudaError_t launch_transfer_H(const DevLevel &fine, int *flag, cudaStream_t s);
cudaError_t launch_coarse_inverse(const DevLevel &L0, double *inv, int64_t n, int *flag,
                                  cudaStream_t s);
cudaError_t launch_assemble_load(const DevLevel &L, const DevOperator &op, double *F, cudaStream_t s);
cudaError_t launch_nu_average(const DevLevel &fine, const double *nu_f, double *nu_c, cudaStream_t s);
cudaError_t launch_adjoint_gradient(int k, const DevLevel &L, const double *ref, const RefTables &rt,
                                    double nu, const double *nu_cell, const double *Lp, const double *La,
                                    const double *rta, double *grad_nu, double *grad_f, cudaStream_t s);
cudaError_t launch_objective(int k, const DevLevel &L, const double *ref, const RefTables &rt, const double *ulat,
                             const double *utgt, double *e_out, double *jcell, cudaStream_t s);
cudaError_t launch_cell_geometry(DevLevel &L, cudaStream_t s);
// post.cu: u* of eq. stPost at the degree-(k+1) lattice from the recovered L_h coefficients and
// u_h lattice values; tabs = P1, P2, P3 packed
cudaError_t launch_poststar(int k, const DevLevel &L, double nu, const double *nu_cell, const double *tabs,
                            int nlat, int npk, const double *Lcoef, const double *ulat, double *out, cudaStream_t s);

// kernels: hot path (ops.cu)
template <class T>
cudaError_t launch_apply(const DevLevel &L, const DevOperator &op, const T *A, const T *x,
                         const T *g, T *y, cudaStream_t s);   // y = A x, or y = g - A x if g
template <class T>
cudaError_t launch_gs_colour(const DevLevel &L, const DevOperator &op, const T *A, const T *Pinv,
                             int colour, const T *g, T *u, cudaStream_t s);
// damped block Jacobi update (eq. bjac) from the residual r = g - A u: every patch's
// correction into D [n_patches][np_max], then u += damping (sum of each unknown's two
// patch corrections); needs L.facet_slot
template <class T>
cudaError_t launch_jacobi_update(const DevLevel &L, const DevOperator &op, const T *Pinv, const T *r, T *D,
                                 double damping, T *u, cudaStream_t s);
// the order-k apply and sweep phase on the 16-bit copies (op.h_fmt), FP32 vectors
cudaError_t launch_apply_h(const DevLevel &L, const DevOperator &op, const float *x, const float *g, float *y,
                           cudaStream_t s);
cudaError_t launch_gs_colour_h(const DevLevel &L, const DevOperator &op, int colour, const float *g, float *u,
                               cudaStream_t s);
// fills op.Pinvp (allocated by the caller) from op.Pinv
cudaError_t launch_pack_sym(const DevLevel &L, DevOperator &op, cudaStream_t s);
// fills op.swQ and op.swA00 (allocated by the caller: n_patches*pc_max*np_max and
// n_patches*pf_max*2 floats) from op.A, op.Pinv and the level's flux weights (2D)
cudaError_t launch_al_split(const DevLevel &L, DevOperator &op, double nu, const double *cell_nu, double gamma,
                            cudaStream_t s);
// fills op.Ah, Ah_s, Pinvh, Pinvh_s (allocated by the caller) from op.A and op.Pinv
cudaError_t launch_round16(const DevLevel &L, DevOperator &op, int fmt, cudaStream_t s);
template <class T>
cudaError_t launch_prolong_add(const DevLevel &fine, const DevLevel &coarse, const T *W,
                               const T *Hm, const T *uc, T *tmp, T *uf, cudaStream_t s);
template <class T>
cudaError_t launch_restrict(const DevLevel &fine, const DevLevel &coarse, const T *W,
                            const T *Hm, const T *rf, T *t1, T *t2, T *rc, cudaStream_t s);
template <class T>
cudaError_t launch_hp_restrict(int k, int64_t n_int, const T *r, T *r0, cudaStream_t s);
template <class T>
cudaError_t launch_hp_prolong_add(int k, int64_t n_int, const T *d0, T *u, cudaStream_t s);
cudaError_t launch_coarse_apply(const double *inv, int64_t n, const double *g, double *u,
                                cudaStream_t s);
template <class T>
cudaError_t launch_mg_small(const SmallParams<T> &S, int l, int m, bool zero_init, size_t smem_per_cta,
                            int cluster_size, cudaStream_t s);
// per-CTA shared memory and cluster size (16/8/4/2 CTAs, 1 = one block, 0 = does not fit)
size_t mg_small_smem(size_t colour_bytes, int csize, int np_max_bytes);
template <class T>
size_t mg_small_vec_bytes(const SmallParams<T> &S, int Ls);
template <class T>
int mg_small_cluster_size(size_t colour_bytes, int np_max_bytes);
cudaError_t launch_d2f(const double *x, float *y, int64_t n, cudaStream_t s);
cudaError_t launch_f2d(const float *x, double *y, int64_t n, cudaStream_t s);
template <class T>
cudaError_t launch_fill(T *x, T v, int64_t n, cudaStream_t s);
cudaError_t launch_axpby(double a, const double *x, double b, double *y, int64_t n, cudaStream_t s);

// Krylov and Uzawa (ops.cu)
int krylov_partial_blocks();
cudaError_t launch_dots(const double *V, int nv, int64_t ld, const double *w, int64_t n,
                        double *partials, cudaStream_t s);
cudaError_t launch_update_dots(const double *V, int nv, int64_t ld, double *w, int64_t n,
                               const double *h, double *partials, int mode, cudaStream_t s);
cudaError_t launch_reduce_partials(const double *partials, int nv, double *out, int accumulate,
                                   cudaStream_t s);
cudaError_t launch_givens(double *small, int j, int restart, double *host_mirror, cudaStream_t s);
cudaError_t launch_scale_next(const double *w, double *v, int64_t n, const double *small, int j,
                              int restart, cudaStream_t s);
cudaError_t launch_init_cycle(const double *r, double *v0, int64_t n, double *small, int restart,
                              cudaStream_t s);
cudaError_t launch_solve_update(double *small, int m, int restart, const double *Z, int64_t ld,
                                double *x, int64_t n, cudaStream_t s);
cudaError_t launch_uzawa_rhs(const DevLevel &L, int k, const double *F, const double *p, double *g,
                             cudaStream_t s);
cudaError_t launch_uzawa_update(const DevLevel &L, int k, const double *u, double *p, double gamma,
                                double nu, const double *nu_cell, const double *bflux, double *partials,
                                cudaStream_t s);
// y = A^T x on a level's FP64 element matrices (non-symmetric operators: Oseen, Newton)
cudaError_t launch_apply_t(const DevLevel &L, const DevOperator &op, const double *x, double *y, cudaStream_t s);
// inhomogeneous Dirichlet data xD [n_boundary][dpf] (finest level, L.cell_bnd): F -= A_IB xD, and
// the per-cell boundary fluxes of the data
cudaError_t launch_dirichlet_load(const DevLevel &L, const DevOperator &op, const double *xD, double *F,
                                  cudaStream_t s);
cudaError_t launch_boundary_flux(const DevLevel &L, int dpf, const double *xD, double *bflux, cudaStream_t s);
cudaError_t launch_sum(const double *x, int64_t n, double *partials, cudaStream_t s);

// multi-right-hand-side kernels (multi.cu): multi-vectors [rows][R], R a power of two <= 64
constexpr int MAX_NRHS = 64;
int krylov_m_blocks();
size_t gs_m_smem(const DevLevel &L, const DevOperator &op, int R, size_t word);
// double-FP32 apply of the order-k operator (A = hi + lo), R columns
cudaError_t launch_apply_df_m(const DevLevel &L, const DevOperator &op, int R, const float *Ahi, const float *Alo,
                              const double *x, float2 *xsplit, const double *g, double *y, cudaStream_t s);
cudaError_t launch_split_lo(const double *A, const float *hi, float *lo, int64_t n, cudaStream_t s);
template <class T>
cudaError_t launch_apply_m(const DevLevel &L, const DevOperator &op, int R, const T *A, const T *x, const T *g, T *y,
                           cudaStream_t s);
// batched order-k colour phase on tensor cores (multi_tc.cu): for operators with 16-bit
// copies (op.h_fmt), dpf = 8 and R in {16, 32, 64}
bool gs_tc_supported(const DevLevel &L, const DevOperator &op, int R);
cudaError_t launch_gs_colour_tc(const DevLevel &L, const DevOperator &op, int R, int colour, const float *g,
                                float *u, cudaStream_t s, int nt = 0);   // nt: threads per block, 128 or 256 (0)
int log2_width(int R);
template <class T>
cudaError_t launch_gs_colour_m(const DevLevel &L, const DevOperator &op, int R, const T *A, const T *Pinv,
                               int colour, const T *g, T *u, cudaStream_t s, int rb = 0, int nt = 0);
                               // rb: rows per thread (divisor of dpf; 0 = default), nt: threads per block (0 = 256)
template <class T>
cudaError_t launch_hp_restrict_m(int k, int64_t n_int, int R, const T *r, T *r0, cudaStream_t s);
template <class T>
cudaError_t launch_hp_prolong_add_m(int k, int64_t n_int, int R, const T *d0, T *u, cudaStream_t s);
template <class T>
cudaError_t launch_prolong_add_m(const DevLevel &F, const DevLevel &C, int R, const T *W, const T *Hm, const T *uc,
                                 T *tmp, T *uf, cudaStream_t s);
template <class T>
cudaError_t launch_restrict_m(const DevLevel &F, const DevLevel &C, int R, const T *W, const T *Hm, const T *rf,
                              T *t1, T *t2, T *rc, cudaStream_t s);
template <class T>
cudaError_t launch_coarse_apply_m(const double *inv, int64_t n, int R, const T *g, T *u, cudaStream_t s);
cudaError_t launch_pack_m(const double *in, int nrhs, int64_t n, int R, double *out, cudaStream_t s);
cudaError_t launch_unpack_m(const double *in, int nrhs, int64_t n, int R, double *out, cudaStream_t s);
template <class Ti, class To>
cudaError_t launch_convert_m(const Ti *x, To *y, int64_t n, cudaStream_t s);
cudaError_t launch_dots_m(const double *V, int nv, int64_t ld, const double *w, int64_t n, int R, double *partials,
                          cudaStream_t s);
cudaError_t launch_update_dots_m(const double *V, int nv, int64_t ld, double *w, int64_t n, int R, const double *h,
                                 double *partials, int mode, cudaStream_t s);
cudaError_t launch_reduce_partials_m(const double *partials, int nv, int R, double *small, int stride, int off,
                                     double *hbuf, cudaStream_t s);
cudaError_t launch_givens_m(double *small, int stride, int j, int Rst, int R, cudaStream_t s);
cudaError_t launch_scale_next_m(const double *w, double *v, int64_t n, int R, const double *small, int stride,
                                int hn_off, cudaStream_t s);
cudaError_t launch_init_cycle_m(const double *r, double *v0, int64_t n, int R, double *small, int stride, int Rst,
                                cudaStream_t s);
cudaError_t launch_solve_update_m(double *small, int stride, const int *m_r, int mmax, int Rst, const double *Z,
                                  int64_t ld, double *x, int64_t n, int R, cudaStream_t s);
cudaError_t launch_uzawa_rhs_m(const DevLevel &L, int k, int R, const double *F, const double *p, double *g,
                               cudaStream_t s);
cudaError_t launch_uzawa_update_m(const DevLevel &L, int k, int R, const double *u, double *p, double gamma, double nu,
                                  const double *nu_cell, const int *frozen, double *partials, cudaStream_t s);

} // namespace hdg
