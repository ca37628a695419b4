// Local post-processing of eq. stPost on the device (triangles; tetrahedra below): u* in [P^{k+1}(K)]^2 with
//   (grad u*, grad v)_K = (-nu^{-1} L_h, grad v)_K  for all v in P^{k+1}(K),
//   (u*, 1)_K = (u_h, 1)_K,
// read with L = -nu grad u so that grad u* approximates grad u (the post-processed
// velocity converges at order k+2 when k >= 1).
//
// One thread per cell.  u* is held by its values at the degree-(k+1) lattice (the
// Lagrange basis lam_n of the forcing layout), so the output has the lattice layout.
// With the affine map x = x0 + J xi, the stiffness is sum_ab G_ab P1[ab] with
// G = |det J| J^{-1} J^{-T}; the Neumann problem's constant null space is closed by the
// rank-one term w w^T, w = 2 P3 (w . 1 = 1), with w . u* = w . u_h on the right: the
// unique solution of the bordered system.  The SPD matrix is factored by Cholesky.
#include <cuda_runtime.h>

#include "hdg3d_internal.h"

namespace hdg {
namespace {

template <int K>
__global__ void __launch_bounds__(128)
poststar_kernel(int64_t nc, const int *__restrict__ cells, const double *__restrict__ coords, double nu,
                const double *__restrict__ nu_cell, const double *__restrict__ P1, const double *__restrict__ P2,
                const double *__restrict__ P3, const double *__restrict__ L, const double *__restrict__ ulat,
                double *__restrict__ out) {
    constexpr int N = (K + 2) * (K + 3) / 2;     // lattice points of degree k+1
    constexpr int NPK = (K + 1) * (K + 2) / 2;
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= nc) return;
    const int v0 = cells[3 * c], v1 = cells[3 * c + 1], v2 = cells[3 * c + 2];
    const double J00 = coords[2 * v1] - coords[2 * v0], J01 = coords[2 * v2] - coords[2 * v0];
    const double J10 = coords[2 * v1 + 1] - coords[2 * v0 + 1], J11 = coords[2 * v2 + 1] - coords[2 * v0 + 1];
    const double det = J00 * J11 - J01 * J10, adet = fabs(det);
    // J^{-1} = [[J11, -J01], [-J10, J00]] / det
    const double Ji[2][2] = {{J11 / det, -J01 / det}, {-J10 / det, J00 / det}};
    double G[2][2];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) G[a][b] = adet * (Ji[a][0] * Ji[b][0] + Ji[a][1] * Ji[b][1]);
    double M[N * (N + 1) / 2];                   // lower triangle, row i at i(i+1)/2
    double w[N];
    for (int i = 0; i < N; ++i) w[i] = 2.0 * P3[i];
    for (int i = 0; i < N; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = w[i] * w[j];
            for (int ab = 0; ab < 4; ++ab) s += G[ab >> 1][ab & 1] * P1[((size_t)ab * N + i) * N + j];
            M[i * (i + 1) / 2 + j] = s;
        }
    // Cholesky in place: M = R R^T, R lower
    for (int j = 0; j < N; ++j) {
        double d = M[j * (j + 1) / 2 + j];
        for (int q = 0; q < j; ++q) d -= M[j * (j + 1) / 2 + q] * M[j * (j + 1) / 2 + q];
        d = sqrt(fmax(d, 1e-300));
        M[j * (j + 1) / 2 + j] = d;
        for (int i = j + 1; i < N; ++i) {
            double s = M[i * (i + 1) / 2 + j];
            for (int q = 0; q < j; ++q) s -= M[i * (i + 1) / 2 + q] * M[j * (j + 1) / 2 + q];
            M[i * (i + 1) / 2 + j] = s / d;
        }
    }
    const double inv_nu = 1.0 / (nu_cell ? nu_cell[c] : nu);
    const double *Lc = L + (size_t)c * 4 * NPK;
    for (int a = 0; a < 2; ++a) {
        // right-hand side: -(1/nu) |det J| sum_{j,d,b} L_{a d, j} (J^{-1})_{b d} P2[j][i][b] + w_i (w . u_h)
        double mean = 0.0;
        for (int n = 0; n < N; ++n) mean += w[n] * ulat[((size_t)c * N + n) * 2 + a];
        double y[N];
        for (int i = 0; i < N; ++i) {
            double s = 0.0;
            for (int j = 0; j < NPK; ++j)
                for (int b = 0; b < 2; ++b) {
                    const double coef = Lc[(2 * a + 0) * NPK + j] * Ji[b][0] + Lc[(2 * a + 1) * NPK + j] * Ji[b][1];
                    s += coef * P2[((size_t)j * N + i) * 2 + b];
                }
            y[i] = -inv_nu * adet * s + w[i] * mean;
        }
        // R y' = y, then R^T x = y'
        for (int i = 0; i < N; ++i) {
            double s = y[i];
            for (int q = 0; q < i; ++q) s -= M[i * (i + 1) / 2 + q] * y[q];
            y[i] = s / M[i * (i + 1) / 2 + i];
        }
        for (int i = N - 1; i >= 0; --i) {
            double s = y[i];
            for (int q = i + 1; q < N; ++q) s -= M[q * (q + 1) / 2 + i] * y[q];
            y[i] = s / M[i * (i + 1) / 2 + i];
        }
        for (int n = 0; n < N; ++n) out[((size_t)c * N + n) * 2 + a] = y[n];
    }
}

// The same on tetrahedra: u* in [P^{k+1}(K)]^3, G = |det J| J^{-1} J^{-T} (3x3), w = 6 P3 (the
// reference volume is 1/6), L_h with the 9 components (c, e) over the orthonormal P^k basis.
template <int K>
__global__ void __launch_bounds__(64)
poststar3_kernel(int64_t nc, const int *__restrict__ cells, const double *__restrict__ coords, double nu,
                 const double *__restrict__ P1, const double *__restrict__ P2, const double *__restrict__ P3,
                 const double *__restrict__ L, const double *__restrict__ ulat, double *__restrict__ out) {
    constexpr int N = (K + 2) * (K + 3) * (K + 4) / 6;
    constexpr int NPK = (K + 1) * (K + 2) * (K + 3) / 6;
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= nc) return;
    double X[4][3];
    for (int v = 0; v < 4; ++v)
        for (int d = 0; d < 3; ++d) X[v][d] = coords[3 * (size_t)cells[4 * c + v] + d];
    double J[3][3];
    for (int r = 0; r < 3; ++r)
        for (int a = 0; a < 3; ++a) J[r][a] = X[a + 1][r] - X[0][r];
    const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                       J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                       J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    const double adet = fabs(det), id = 1.0 / det;
    double Ji[3][3];
    Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) * id;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
    Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) * id;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
    Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) * id;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
    double G[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) G[a][b] = adet * (Ji[a][0] * Ji[b][0] + Ji[a][1] * Ji[b][1] + Ji[a][2] * Ji[b][2]);
    double M[N * (N + 1) / 2];
    double w[N];
    for (int i = 0; i < N; ++i) w[i] = 6.0 * P3[i];
    for (int i = 0; i < N; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = w[i] * w[j];
            for (int ab = 0; ab < 9; ++ab) s += G[ab / 3][ab % 3] * P1[((size_t)ab * N + i) * N + j];
            M[i * (i + 1) / 2 + j] = s;
        }
    for (int j = 0; j < N; ++j) {
        double d = M[j * (j + 1) / 2 + j];
        for (int q = 0; q < j; ++q) d -= M[j * (j + 1) / 2 + q] * M[j * (j + 1) / 2 + q];
        d = sqrt(fmax(d, 1e-300));
        M[j * (j + 1) / 2 + j] = d;
        for (int i = j + 1; i < N; ++i) {
            double s = M[i * (i + 1) / 2 + j];
            for (int q = 0; q < j; ++q) s -= M[i * (i + 1) / 2 + q] * M[j * (j + 1) / 2 + q];
            M[i * (i + 1) / 2 + j] = s / d;
        }
    }
    const double *Lc = L + (size_t)c * 9 * NPK;
    for (int a = 0; a < 3; ++a) {
        double mean = 0.0;
        for (int n = 0; n < N; ++n) mean += w[n] * ulat[((size_t)c * N + n) * 3 + a];
        double y[N];
        for (int i = 0; i < N; ++i) {
            double s = 0.0;
            for (int j = 0; j < NPK; ++j)
                for (int b = 0; b < 3; ++b) {
                    const double coef = Lc[(3 * a + 0) * NPK + j] * Ji[b][0] + Lc[(3 * a + 1) * NPK + j] * Ji[b][1] +
                                        Lc[(3 * a + 2) * NPK + j] * Ji[b][2];
                    s += coef * P2[((size_t)j * N + i) * 3 + b];
                }
            y[i] = -adet * s / nu + w[i] * mean;
        }
        for (int i = 0; i < N; ++i) {
            double s = y[i];
            for (int q = 0; q < i; ++q) s -= M[i * (i + 1) / 2 + q] * y[q];
            y[i] = s / M[i * (i + 1) / 2 + i];
        }
        for (int i = N - 1; i >= 0; --i) {
            double s = y[i];
            for (int q = i + 1; q < N; ++q) s -= M[q * (q + 1) / 2 + i] * y[q];
            y[i] = s / M[i * (i + 1) / 2 + i];
        }
        for (int n = 0; n < N; ++n) out[((size_t)c * N + n) * 3 + a] = y[n];
    }
}

} // namespace

cudaError_t launch_poststar(int k, const DevLevel &L, double nu, const double *nu_cell, const double *tabs,
                            int nlat, int npk, const double *Lcoef, const double *ulat, double *out, cudaStream_t s) {
    if (L.nc == 0) return cudaSuccess;
    const double *P1 = tabs, *P2 = P1 + (size_t)4 * nlat * nlat, *P3 = P2 + (size_t)npk * nlat * 2;
    const unsigned nb = (unsigned)((L.nc + 127) / 128);
    note_launches(1);
    switch (k) {
#define HDG_POST(K)                                                                                              \
    case K:                                                                                                      \
        poststar_kernel<K><<<nb, 128, 0, s>>>(L.nc, L.cells.p, L.coords.p, nu, nu_cell, P1, P2, P3, Lcoef, ulat, \
                                              out);                                                              \
        break;
        HDG_POST(0) HDG_POST(1) HDG_POST(2) HDG_POST(3) HDG_POST(4)
#undef HDG_POST
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_poststar3(int k, const DevLevel &L, double nu, const double *tabs, int nlat, int npk,
                             const double *Lcoef, const double *ulat, double *out, cudaStream_t s) {
    if (L.nc == 0) return cudaSuccess;
    const double *P1 = tabs, *P2 = P1 + (size_t)9 * nlat * nlat, *P3 = P2 + (size_t)npk * nlat * 3;
    const unsigned nb = (unsigned)((L.nc + 63) / 64);
    note_launches(1);
    switch (k) {
#define HDG_POST3(K)                                                                                          \
    case K:                                                                                                   \
        poststar3_kernel<K><<<nb, 64, 0, s>>>(L.nc, L.cells.p, L.coords.p, nu, P1, P2, P3, Lcoef, ulat, out); \
        break;
        HDG_POST3(0) HDG_POST3(1) HDG_POST3(2) HDG_POST3(3)
#undef HDG_POST3
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

} // namespace hdg
