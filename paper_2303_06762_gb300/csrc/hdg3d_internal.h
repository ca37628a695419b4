// Internal declarations of the 3D (tetrahedral) path.
//
// The 3D path shares the context, the device level structure, the Krylov and Uzawa
// drivers and the multigrid recursion with 2D; what differs lives here: the host
// topology of tetrahedral levels (faces, edge patches, the transfer slots of Bey's
// red refinement), the reference-tetrahedron tables and the kernels that know four
// faces per cell and three lowest-order unknowns per face.
#pragma once

#include <array>
#include <string>
#include <vector>

#include "hdg_internal.h"

namespace hdg {

// reference3d.cpp
void build_reference_tables_3d(int k, RefTables3 &out);
std::vector<double> pack_reference_tables_3d(const RefTables3 &t);   // R1..R6, Q, FA consecutive

// topology3d.cpp
std::string build_level_topology_3d(HostLevel3 &L);
std::string build_transfer_3d(const HostLevel3 &coarse, const HostLevel3 &fine, HostTransfer3 &T);

// condense3d.cu: element matrices (with the AL term), flux weights, volumes and element loads
// of one tetrahedral level; scratch: device workspace of condense3_scratch_doubles(k) doubles
size_t condense3_scratch_doubles(int k, int blocks);
// recovery mode (x non-null): the cell unknowns of the skeleton solution x [n_int][dpf] instead of
// the element matrices and loads: RT coefficients in the reference basis rt [nc][nrt], L_h over the
// orthonormal P^k basis L [nc][9][npk] (components xx, xy, xz, yx, ..., zz), u_h at the lattice
// ulat [nc][nlat][3] (each output nullable)
struct Recover3 {
    const double *x = nullptr;
    const int *cell_int = nullptr;
    const int *cell_bnd = nullptr;    // with xD: boundary face number of each local face or -1
    const double *xD = nullptr;       // Dirichlet data [n_boundary][dpf], or null (homogeneous)
    double *rt = nullptr, *L = nullptr, *ulat = nullptr;
};
cudaError_t launch_condense3(int k, const DevLevel &L, const double *ref, const RefTables3 &rt, double nu,
                             const double *nu_cell, double beta, double gamma, const double *forcing, double *A,
                             float *Af, double *Fel, double *scratch, int blocks, int *flag, cudaStream_t s,
                             const Recover3 &rec = Recover3());
cudaError_t launch_transfer_H3(const DevLevel &fine, int *flag, cudaStream_t s);
// edge-patch inverses with the patch matrices in a global workspace (blocks slices of np_max^2)
size_t patch_inverse3_scratch_doubles(const DevLevel &L, const DevOperator &op, int blocks);
cudaError_t launch_patch_inverse3(const DevLevel &L, const DevOperator &op, double *scratch, int blocks, int *flag,
                                  cudaStream_t s);

// post.cu: u* of eq. stPost on tetrahedra at the degree-(k+1) lattice; tabs = P1, P2, P3 packed
cudaError_t launch_poststar3(int k, const DevLevel &L, double nu, const double *tabs, int nlat, int npk,
                             const double *Lcoef, const double *ulat, double *out, cudaStream_t s);

// ops3d.cu: hot-path kernels with four faces per cell
template <class T>
cudaError_t launch_apply3(const DevLevel &L, int dpf, const T *A, const T *x, const T *g, T *y, cudaStream_t s);
template <class T>
cudaError_t launch_gs_colour3(const DevLevel &L, const DevOperator &op, const T *A, const T *Pinv, int colour,
                              const T *g, T *u, cudaStream_t s);
template <class T>
cudaError_t launch_prolong_add3(const DevLevel &fine, const DevLevel &coarse, const T *W, const T *Hm, const T *uc,
                                T *tmp, T *uf, cudaStream_t s);
template <class T>
cudaError_t launch_restrict3(const DevLevel &fine, const DevLevel &coarse, const T *W, const T *Hm, const T *rf,
                             T *t1, T *t2, T *rc, cudaStream_t s);
template <class T>
cudaError_t launch_hp_restrict3(int k, int64_t n_int, const T *r, T *r0, cudaStream_t s);
template <class T>
cudaError_t launch_hp_prolong_add3(int k, int64_t n_int, const T *d0, T *u, cudaStream_t s);

} // namespace hdg
