// Device-side setup in FP64: static condensation, patch inverses, harmonic
// extension blocks, coarsest dense inverse, element geometry and loads.
//
// Static condensation (Section 3.2): on every cell the local system of
// eq. stWeak is formed from reference tables (reference.cpp) and the
// element Jacobian J: with the Piola map phi = J phi^/det J the tensor
// C(G; u, û) = (∇u, G) − <tng u, G n> + <tng û, G n> is a contraction of the
// reference integrals R1, R2, R3; the mass, divergence and load blocks are
// contractions of R4, R5, R6.  The flux L is eliminated in closed form
// (orthonormal P^k basis: mass ν⁻¹|det J| I), leaving
//     K = (ν/|det J|) CᵀC + β M_u     on (u, û).
// The interior RT unknowns u_i and the mean-free pressure p_o are then
// eliminated by block Cholesky:
//     Y = K_ii⁻¹[K_ig | D_oiᵀ | F_i],  S_p = D_oi Y_D,  W = D_oi Y_g − D_og,
//     A_K = K_gg − K_gi Y_g + Wᵀ S_p⁻¹ W,
//     F_K = F_g − K_gi Y_F + Wᵀ S_p⁻¹ D_oi Y_F,
// and the augmented-Lagrangian term ε⁻¹|K|⁻¹ d dᵀ (eq. stALform; d = the
// cell's flux functional) is added.
// Oseen (Section 4.1): with a convecting field w_h the upwind form
//     −(u, (w·∇)v)_K + ⟨(w·n)⁺ tng u + (w·n)⁻ tng û, tng(v − v̂)⟩_∂K
// is added to K from point values (tables R9–R16; the facet switch is taken
// at the Gauss–Legendre nodes).  K is then non-symmetric, the two
// eliminations use LU with partial pivoting, and with W₂ = K_gi Y_D − D_ogᵀ
// in place of Wᵀ:
//     A_K = K_gg − K_gi Y_g + W₂ S_p⁻¹ W,   F_K = F_g − K_gi Y_F + W₂ S_p⁻¹ D_oi Y_F.
// With conv_t the transposed convection block is used (the adjoint system).
// A Newton step (Section 4.2, Algorithm 3) adds the derivative of the upwind
// form in its convecting argument, with the switch frozen at u_old·n_K, and
// the load C_h(u_old; u_old, v) on the (u, û) rows (newton_x = the previous
// skeleton iterate, conv = u_old at the lattice).
// Element matrices are stored by row blocks: the DPF rows of local facet f form
// one contiguous block [f][column][row within the facet], so that a facet's rows
// (what the apply and the smoothers read) are one contiguous DPF·n_loc stretch
// and the DPF threads of a facet read consecutive addresses.  Facet unknowns are expressed in the
// global facet basis of include/hdg.h: the reference facet moments map to
// the global ones by the factor sqrt|F|·σ·sgn(det J)·o^m (σ = n_F·n_K,
// o = ±1 the orientation of the facet parameter).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>

#include "hdg3d_internal.h"

namespace hdg {
namespace {

__constant__ int c_FV[3][2] = {{1, 2}, {0, 2}, {0, 1}};

template <int K>
struct Dims {
    static constexpr int NPK = (K + 1) * (K + 2) / 2;
    static constexpr int NRT = (K + 1) * (K + 3);
    static constexpr int NF = K + 1;
    static constexpr int NL = 4 * NPK;
    static constexpr int NCOL = NRT + 3 * NF;
    static constexpr int NG = 6 * NF;
    static constexpr int NRI = K * (K + 1);
    static constexpr int NPO = NPK - 1;
    static constexpr int NLAT = (K + 2) * (K + 3) / 2;
    static constexpr int NY = NG + NPO + 1;
    // shared memory layout (doubles)
    static constexpr int O_GEO = 0;                    // 64 doubles of geometry
    static constexpr int O_S = 64;                     // NRT facet scaling
    static constexpr int O_C = O_S + NRT;
    static constexpr int O_K = O_C + NL * NCOL;
    static constexpr int O_D = O_K + NCOL * NCOL;
    static constexpr int O_F = O_D + NRT * NPK;
    static constexpr int O_FN = O_F + NCOL;                // load over all (u, û) rows
    static constexpr int O_Y = O_FN + 2 * NLAT;
    static constexpr int O_SP = O_Y + NRI * NY;
    static constexpr int O_W = O_SP + NPO * NPO;
    static constexpr int O_Z = O_W + NPO * NG;
    static constexpr int O_LII = O_Z + NPO * (NG + 1);
    static constexpr int O_XG = O_LII + NRI * NRI;       // recovery: gathered skeleton values
    static constexpr int O_XF = O_XG + NG;                // recovery: all (u, û) coefficients
    static constexpr int O_PO = O_XF + NCOL;              // recovery: mean-free pressure
    static constexpr int TOTAL = O_PO + NPO + 1;
    // convection (only when a field is given)
    static constexpr int NQ = (K + 5) * (K + 5);           // volume nodes
    static constexpr int NFQ = (3 * K + 5) / 2;            // nodes per facet
    static constexpr int O_W2 = TOTAL;                     // W2 (NPO x NG, stored [j][p])
    static constexpr int O_WL = O_W2 + NPO * NG;           // lattice values of w
    static constexpr int O_WH = O_WL + 2 * NLAT;           // J^{-1} w at volume nodes
    static constexpr int O_GQ = O_WH + 2 * NQ;             // weight * (w^·∇^) phi^_i
    static constexpr int O_HQ = O_GQ + NQ * NRT * 2;       // JᵀJ phi^_j
    static constexpr int O_TAU = O_HQ + NQ * NRT * 2;      // tangential traces at facet nodes
    static constexpr int O_AW = O_TAU + 3 * NFQ * NCOL;    // |F| weight (w·n_K) at facet nodes
    static constexpr int TOTAL_CONV = O_AW + 3 * NFQ;
    // Newton term (only with a previous skeleton iterate); G2 reuses the GQ region, which
    // the Picard part no longer needs when the Newton part starts
    static constexpr int O_G2 = O_GQ;                       // weight (Jᵀu_old)·∇^ phi^_i at volume nodes
    static constexpr int O_NRM = TOTAL_CONV;                // phi_j·n_K at facet nodes
    static constexpr int O_WUP = O_NRM + 3 * NFQ * NRT;     // upwinded tangential u_old at facet nodes
    static constexpr int O_UH = O_WUP + 3 * NFQ;            // û_old tangential coefficients (3 x NF)
    static constexpr int TOTAL_NEWTON = O_UH + 3 * NF;
};

// geometry slots inside the O_GEO block
enum { G_J = 0, G_JI = 4, G_DET = 8, G_SGN = 9, G_LEN = 10, G_NK = 13, G_TF = 19, G_SIG = 25,
       G_O = 28, G_AREA = 31 };

__device__ void cell_geometry(const double *coords, const int *cells, int64_t c, double *geo) {
    int v[3];
    double X[3][2];
    for (int i = 0; i < 3; ++i) {
        v[i] = cells[3 * c + i];
        X[i][0] = coords[2 * v[i]];
        X[i][1] = coords[2 * v[i] + 1];
    }
    double J00 = X[1][0] - X[0][0], J01 = X[2][0] - X[0][0];
    double J10 = X[1][1] - X[0][1], J11 = X[2][1] - X[0][1];
    double det = J00 * J11 - J01 * J10;
    geo[G_J + 0] = J00; geo[G_J + 1] = J01; geo[G_J + 2] = J10; geo[G_J + 3] = J11;
    geo[G_JI + 0] = J11 / det; geo[G_JI + 1] = -J01 / det;
    geo[G_JI + 2] = -J10 / det; geo[G_JI + 3] = J00 / det;
    geo[G_DET] = det;
    geo[G_SGN] = det > 0 ? 1.0 : -1.0;
    geo[G_AREA] = 0.5 * fabs(det);
    for (int f = 0; f < 3; ++f) {
        int a = c_FV[f][0], b = c_FV[f][1];
        double dx = X[b][0] - X[a][0], dy = X[b][1] - X[a][1];
        double len = sqrt(dx * dx + dy * dy);
        double o = v[a] < v[b] ? 1.0 : -1.0;
        double tx = o * dx / len, ty = o * dy / len;
        double nx = ty, ny = -tx;
        double mx = 0.5 * (X[a][0] + X[b][0]) - X[f][0], my = 0.5 * (X[a][1] + X[b][1]) - X[f][1];
        double sig = (nx * mx + ny * my) > 0 ? 1.0 : -1.0;
        geo[G_LEN + f] = len;
        geo[G_NK + 2 * f] = sig * nx; geo[G_NK + 2 * f + 1] = sig * ny;
        geo[G_TF + 2 * f] = tx; geo[G_TF + 2 * f + 1] = ty;
        geo[G_SIG + f] = sig;
        geo[G_O + f] = o;
    }
}

// in-place Cholesky of the n x n matrix in sm (row-major, leading dim ld), serial;
// returns false on a non-positive pivot
__device__ bool chol_serial(double *sm, int n, int ld) {
    for (int j = 0; j < n; ++j) {
        double d = sm[j * ld + j];
        for (int p = 0; p < j; ++p) d -= sm[j * ld + p] * sm[j * ld + p];
        if (!(d > 0.0)) return false;
        d = sqrt(d);
        sm[j * ld + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double s = sm[i * ld + j];
            for (int p = 0; p < j; ++p) s -= sm[i * ld + p] * sm[j * ld + p];
            sm[i * ld + j] = s / d;
        }
    }
    return true;
}

// in-place LU factorisation with partial pivoting (unit lower L), serial: row j
// of the factors is row perm[j] swapped in at step j; returns false on a zero or
// non-finite pivot
__device__ bool lu_serial(double *sm, int n, int ld, int *perm) {
    for (int j = 0; j < n; ++j) {
        int p = j;
        double best = fabs(sm[j * ld + j]);
        for (int i = j + 1; i < n; ++i)
            if (fabs(sm[i * ld + j]) > best) {
                best = fabs(sm[i * ld + j]);
                p = i;
            }
        perm[j] = p;
        if (!(best > 1e-300) || !isfinite(best)) return false;
        if (p != j)
            for (int c = 0; c < n; ++c) {
                const double t = sm[j * ld + c];
                sm[j * ld + c] = sm[p * ld + c];
                sm[p * ld + c] = t;
            }
        const double d = sm[j * ld + j];
        for (int i = j + 1; i < n; ++i) {
            const double l = sm[i * ld + j] / d;
            sm[i * ld + j] = l;
            for (int c = j + 1; c < n; ++c) sm[i * ld + c] -= l * sm[j * ld + c];
        }
    }
    return true;
}

// solve (LU) x = P b for column `col` of the row-major RHS block B (n x nb, ld ldb)
__device__ void lu_solve_col(const double *LU, int n, int ld, const int *perm, double *B, int ldb, int col) {
    for (int j = 0; j < n; ++j) {
        const int p = perm[j];
        if (p != j) {
            const double t = B[j * ldb + col];
            B[j * ldb + col] = B[p * ldb + col];
            B[p * ldb + col] = t;
        }
    }
    for (int i = 0; i < n; ++i) {
        double s = B[i * ldb + col];
        for (int p = 0; p < i; ++p) s -= LU[i * ld + p] * B[p * ldb + col];
        B[i * ldb + col] = s;
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = B[i * ldb + col];
        for (int p = i + 1; p < n; ++p) s -= LU[i * ld + p] * B[p * ldb + col];
        B[i * ldb + col] = s / LU[i * ld + i];
    }
}

// solve L Lᵀ x = b for column `col` of the row-major RHS block B (n x nb, ld ldb)
__device__ void chol_solve_col(const double *Lm, int n, int ld, double *B, int ldb, int col) {
    for (int i = 0; i < n; ++i) {
        double s = B[i * ldb + col];
        for (int p = 0; p < i; ++p) s -= Lm[i * ld + p] * B[p * ldb + col];
        B[i * ldb + col] = s / Lm[i * ld + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = B[i * ldb + col];
        for (int p = i + 1; p < n; ++p) s -= Lm[p * ld + i] * B[p * ldb + col];
        B[i * ldb + col] = s / Lm[i * ld + i];
    }
}

struct RefPtrs {
    const double *R[N_REF_TABLES];
};

// Upwind convection of Section 4.1 on the (u, û) block of K (rows = test
// functions, columns = trial functions, the basis of Km), added to Km; with
// conv_t its transpose is added instead.
//   volume:  −(sc_i sc_j/|det J|) Σ_q ω_q (ŵ·∇̂ φ̂_i)ᵀ JᵀJ φ̂_j,   ŵ = J⁻¹ w
//   facets:  |F| ω_g (w·n_K) at node g switches between the traces of u (w·n_K > 0)
//            and û (w·n_K < 0); tangential traces t_F·φ_i = o sc_i t̂ᵀJᵀJ φ̂_i/(|F| det J)
//            and, for û, o^m l_m(s_g)/sqrt|F|.
template <int K>
__device__ void convection_block(int64_t c, const double *__restrict__ conv, int conv_t,
                                 const double *__restrict__ newton_x, const int *__restrict__ cell_int,
                                 const RefPtrs &T, const double *geo, const double *sc, double *Km, double *Fl,
                                 double *sm) {
    using D = Dims<K>;
    const double *__restrict__ R9 = T.R[8];
    const double *__restrict__ R10 = T.R[9];
    const double *__restrict__ R11 = T.R[10];
    const double *__restrict__ R12 = T.R[11];
    const double *__restrict__ R13 = T.R[12];
    const double *__restrict__ R14 = T.R[13];
    const double *__restrict__ R15 = T.R[14];
    const double *__restrict__ R16 = T.R[15];
    double *wl = sm + D::O_WL, *wh = sm + D::O_WH, *Gq = sm + D::O_GQ, *Hq = sm + D::O_HQ;
    double *tau = sm + D::O_TAU, *aw = sm + D::O_AW;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int i = tid; i < 2 * D::NLAT; i += nt) wl[i] = conv[c * 2 * D::NLAT + i];
    __syncthreads();
    const double det = geo[G_DET], adet = fabs(det);
    for (int q = tid; q < D::NQ; q += nt) {
        double wx = 0.0, wy = 0.0;
        for (int n = 0; n < D::NLAT; ++n) {
            const double l = R11[q * D::NLAT + n];
            wx += l * wl[2 * n];
            wy += l * wl[2 * n + 1];
        }
        wh[2 * q] = geo[G_JI + 0] * wx + geo[G_JI + 1] * wy;
        wh[2 * q + 1] = geo[G_JI + 2] * wx + geo[G_JI + 3] * wy;
    }
    for (int fg = tid; fg < 3 * D::NFQ; fg += nt) {
        const int f = fg / D::NFQ, g = fg % D::NFQ;
        double wx = 0.0, wy = 0.0;
        for (int n = 0; n < D::NLAT; ++n) {
            const double l = R14[fg * D::NLAT + n];
            wx += l * wl[2 * n];
            wy += l * wl[2 * n + 1];
        }
        aw[fg] = geo[G_LEN + f] * R16[g] * (wx * geo[G_NK + 2 * f] + wy * geo[G_NK + 2 * f + 1]);
    }
    __syncthreads();
    double JtJ[4];
    JtJ[0] = geo[G_J + 0] * geo[G_J + 0] + geo[G_J + 2] * geo[G_J + 2];
    JtJ[1] = geo[G_J + 0] * geo[G_J + 1] + geo[G_J + 2] * geo[G_J + 3];
    JtJ[2] = JtJ[1];
    JtJ[3] = geo[G_J + 1] * geo[G_J + 1] + geo[G_J + 3] * geo[G_J + 3];
    for (int idx = tid; idx < D::NQ * D::NRT * 2; idx += nt) {
        const int a = idx & 1, qi = idx >> 1, q = qi / D::NRT;
        const double *d = R10 + (size_t)idx * 2;
        Gq[idx] = R12[q] * (wh[2 * q] * d[0] + wh[2 * q + 1] * d[1]);
        const double *ph = R9 + (size_t)qi * 2;
        Hq[idx] = JtJ[2 * a] * ph[0] + JtJ[2 * a + 1] * ph[1];
    }
    for (int idx = tid; idx < 3 * D::NFQ * D::NCOL; idx += nt) {
        const int fg = idx / D::NCOL, col = idx % D::NCOL, f = fg / D::NFQ, g = fg % D::NFQ;
        double v = 0.0;
        if (col < D::NRT) {
            const double *ph = R13 + ((size_t)fg * D::NRT + col) * 2;
            // reference edge vector of facet f (from its lower to its higher local vertex)
            const double tx = f == 0 ? -1.0 : (f == 1 ? 0.0 : 1.0);
            const double ty = f == 2 ? 0.0 : 1.0;
            const double j0 = JtJ[0] * ph[0] + JtJ[1] * ph[1], j1 = JtJ[2] * ph[0] + JtJ[3] * ph[1];
            v = sc[col] * geo[G_O + f] / (geo[G_LEN + f] * det) * (tx * j0 + ty * j1);
        } else {
            const int h = col - D::NRT, f2 = h / D::NF, m = h % D::NF;
            if (f2 == f) v = ((m & 1) ? geo[G_O + f] : 1.0) * R15[g * D::NF + m] / sqrt(geo[G_LEN + f]);
        }
        tau[idx] = v;
    }
    __syncthreads();
    for (int idx = tid; idx < D::NCOL * D::NCOL; idx += nt) {
        const int r = idx / D::NCOL, s2 = idx % D::NCOL;
        const int i = conv_t ? s2 : r, j = conv_t ? r : s2;
        double v = 0.0;
        if (i < D::NRT && j < D::NRT) {
            double acc = 0.0;
            for (int q = 0; q < D::NQ; ++q) {
                const double *gi = Gq + (q * D::NRT + i) * 2, *hj = Hq + (q * D::NRT + j) * 2;
                acc += gi[0] * hj[0] + gi[1] * hj[1];
            }
            v = -sc[i] * sc[j] / adet * acc;
        }
        for (int fg = 0; fg < 3 * D::NFQ; ++fg) {
            const double a = aw[fg];
            const double ap = a > 0.0 ? a : 0.0, am = a < 0.0 ? a : 0.0;
            const double coef = i < D::NRT ? (j < D::NRT ? ap : am) : (j < D::NRT ? -ap : -am);
            v += coef * tau[fg * D::NCOL + i] * tau[fg * D::NCOL + j];
        }
        Km[idx] += v;
    }
    __syncthreads();
    if (!newton_x) return;
    // Newton term of Algorithm 3 (derivative of the upwind form in its convecting argument, the
    // switch frozen at u_old·n_K), on rows (v, v̂) and columns δu:
    //   -(u_old, (φ_j·∇)φ_i) + <(φ_j·n_K) u_old^up, tng(v - v̂)>,
    // and the load C_h(u_old; u_old, v) (the same form at δu = u_old), with u_old = w (lattice
    // values) and u_old^up = tng u_old where u_old·n_K > 0, tng û_old elsewhere.
    double *G2 = sm + D::O_G2, *nrm = sm + D::O_NRM, *wup = sm + D::O_WUP, *uh = sm + D::O_UH;
    __shared__ double s_tie;
    if (tid == 0) {
        double mx = 0.0;
        for (int i = 0; i < 2 * D::NLAT; ++i) mx = fmax(mx, fabs(wl[i]));
        s_tie = 1e-10 * mx;     // |w·n| at rounding level counts as zero (same rule as the oracle)
    }
    for (int i = tid; i < 3 * D::NF; i += nt) {
        const int f = i / D::NF, m = i % D::NF;
        const int j = cell_int[3 * c + f];
        uh[i] = j >= 0 ? newton_x[(size_t)j * 2 * D::NF + D::NF + m] : 0.0;
    }
    for (int idx = tid; idx < D::NQ * D::NRT * 2; idx += nt) {
        // G2[q][i][b] = ω_q Σ_a (Jᵀ u_old)_a d_b phi^_{i,a}
        const int b = idx & 1, qi = idx >> 1, q = qi / D::NRT, i = qi % D::NRT;
        double wx = 0.0, wy = 0.0;
        for (int n = 0; n < D::NLAT; ++n) {
            const double l = R11[q * D::NLAT + n];
            wx += l * wl[2 * n];
            wy += l * wl[2 * n + 1];
        }
        const double t0 = geo[G_J + 0] * wx + geo[G_J + 2] * wy, t1 = geo[G_J + 1] * wx + geo[G_J + 3] * wy;
        const double *d = R10 + ((size_t)(q * D::NRT + i) * 2) * 2;   // [a][b]
        G2[idx] = R12[q] * (t0 * d[0 * 2 + b] + t1 * d[1 * 2 + b]);
    }
    for (int idx = tid; idx < 3 * D::NFQ * D::NRT; idx += nt) {
        const int fg = idx / D::NRT, j = idx % D::NRT, f = fg / D::NFQ;
        const double *ph = R13 + ((size_t)fg * D::NRT + j) * 2;
        const double px = geo[G_J + 0] * ph[0] + geo[G_J + 1] * ph[1], py = geo[G_J + 2] * ph[0] + geo[G_J + 3] * ph[1];
        nrm[idx] = sc[j] * (px * geo[G_NK + 2 * f] + py * geo[G_NK + 2 * f + 1]) / det;
    }
    __syncthreads();
    for (int fg = tid; fg < 3 * D::NFQ; fg += nt) {
        const int f = fg / D::NFQ;
        double wx = 0.0, wy = 0.0;
        for (int n = 0; n < D::NLAT; ++n) {
            const double l = R14[fg * D::NLAT + n];
            wx += l * wl[2 * n];
            wy += l * wl[2 * n + 1];
        }
        double v;
        // ties: where |w·n| is at rounding level (Dirichlet facets, symmetric nodes) the
        // trace of û is taken, so the switch does not follow rounding noise
        const double wn = wx * geo[G_NK + 2 * f] + wy * geo[G_NK + 2 * f + 1];
        if (wn > s_tie && cell_int[3 * c + f] >= 0) {
            v = wx * geo[G_TF + 2 * f] + wy * geo[G_TF + 2 * f + 1];
        } else {
            v = 0.0;
            for (int m = 0; m < D::NF; ++m) v += uh[f * D::NF + m] * tau[fg * D::NCOL + D::NRT + f * D::NF + m];
        }
        wup[fg] = v;
    }
    __syncthreads();
    for (int idx = tid; idx < D::NCOL * D::NRT; idx += nt) {
        const int row = idx / D::NRT, j = idx % D::NRT;
        double v = 0.0;
        if (row < D::NRT) {
            double acc = 0.0;
            for (int q = 0; q < D::NQ; ++q) {
                const double *g2 = G2 + (q * D::NRT + row) * 2;
                const double *ph = R9 + ((size_t)q * D::NRT + j) * 2;
                acc += g2[0] * ph[0] + g2[1] * ph[1];
            }
            v = -sc[row] * sc[j] / adet * acc;
        }
        const double sr = row < D::NRT ? 1.0 : -1.0;
        for (int fg = 0; fg < 3 * D::NFQ; ++fg) {
            const int f = fg / D::NFQ, g = fg % D::NFQ;
            const double lw = geo[G_LEN + f] * R16[g];
            v += sr * lw * nrm[fg * D::NRT + j] * wup[fg] * tau[fg * D::NCOL + row];
        }
        Km[row * D::NCOL + j] += v;
    }
    for (int row = tid; row < D::NCOL; row += nt) {
        double v = 0.0;
        if (row < D::NRT) {
            double acc = 0.0;
            for (int q = 0; q < D::NQ; ++q) {
                const double *g2 = G2 + (q * D::NRT + row) * 2;
                acc += g2[0] * wh[2 * q] + g2[1] * wh[2 * q + 1];
            }
            v = -sc[row] * (det > 0.0 ? 1.0 : -1.0) * acc;
        }
        const double sr = row < D::NRT ? 1.0 : -1.0;
        for (int fg = 0; fg < 3 * D::NFQ; ++fg) v += sr * aw[fg] * wup[fg] * tau[fg * D::NCOL + row];
        Fl[row] += v;
    }
    __syncthreads();
}

template <int K>
__global__ void __launch_bounds__(128)
condense_kernel(int64_t nc, const double *__restrict__ coords, const int *__restrict__ cells,
                RefPtrs T, double nu_scalar, const double *__restrict__ nu_cell,
                double beta, double gamma, const double *__restrict__ forcing,
                const double *__restrict__ conv, int conv_t, const double *__restrict__ newton_x,
                const int *__restrict__ cell_int,
                double *__restrict__ Aout, float *__restrict__ Afout, double *__restrict__ Fout,
                int *flag, RecoverArgs rec) {
    using D = Dims<K>;
    const double *__restrict__ R1 = T.R[0];
    const double *__restrict__ R2 = T.R[1];
    const double *__restrict__ R3 = T.R[2];
    const double *__restrict__ R4 = T.R[3];
    const double *__restrict__ R5 = T.R[4];
    const double *__restrict__ R6 = T.R[5];
    const double *__restrict__ R7 = T.R[6];
    extern __shared__ double sm[];
    double *geo = sm + D::O_GEO;
    double *sc = sm + D::O_S;
    double *C = sm + D::O_C;
    double *Km = sm + D::O_K;
    double *Dm = sm + D::O_D;
    double *Fl = sm + D::O_F;
    double *Fn = sm + D::O_FN;
    double *Y = sm + D::O_Y;
    double *Sp = sm + D::O_SP;
    double *Wm = sm + D::O_W;
    double *Zm = sm + D::O_Z;
    double *Lii = sm + D::O_LII;
    double *xg = sm + D::O_XG;
    double *xf = sm + D::O_XF;
    double *po = sm + D::O_PO;
    double *W2 = sm + D::O_W2;
    const int tid = threadIdx.x, nt = blockDim.x;
    __shared__ int s_ok;
    __shared__ int s_perm[32];   // row interchanges of the LU factorisations (NRI, NPO <= 20)

    for (int64_t c = blockIdx.x; c < nc; c += gridDim.x) {
        if (tid == 0) {
            cell_geometry(coords, cells, c, geo);
            s_ok = 1;
        }
        if (forcing)
            for (int i = tid; i < 2 * D::NLAT; i += nt) Fn[i] = forcing[c * 2 * D::NLAT + i];
        __syncthreads();
        const double det = geo[G_DET], sgn = geo[G_SGN], adet = fabs(det);
        const double nu = nu_cell ? nu_cell[c] : nu_scalar;
        const double eps_inv = gamma * nu;
        for (int i = tid; i < D::NRT; i += nt) {
            double s = 1.0;
            if (i < 3 * D::NF) {
                int f = i / D::NF, m = i % D::NF;
                s = sqrt(geo[G_LEN + f]) * geo[G_SIG + f] * sgn * ((m & 1) ? geo[G_O + f] : 1.0);
            }
            sc[i] = s;
        }
        __syncthreads();
        // C = [C_u | C_hat], rows (c, e, j) with flux component (c, e) and g_j
        for (int idx = tid; idx < D::NL * D::NCOL; idx += nt) {
            int row = idx / D::NCOL, col = idx % D::NCOL;
            int ce = row / D::NPK, j = row % D::NPK, cc = ce >> 1, e = ce & 1;
            double val;
            if (col < D::NRT) {
                int i = col;
                double vol = 0.0;
                for (int a = 0; a < 2; ++a)
                    for (int b = 0; b < 2; ++b)
                        vol += geo[G_J + 2 * cc + a] * geo[G_JI + 2 * b + e] *
                               R1[((i * 2 + a) * 2 + b) * D::NPK + j];
                vol *= sgn;
                double bnd = 0.0;
                const double fl[3] = {1.4142135623730951, 1.0, 1.0};
                for (int f = 0; f < 3; ++f) {
                    double nx = geo[G_NK + 2 * f], ny = geo[G_NK + 2 * f + 1];
                    double ne = e == 0 ? nx : ny, nc_ = cc == 0 ? nx : ny;
                    double acc = 0.0;
                    for (int a = 0; a < 2; ++a) {
                        double nJ = nx * geo[G_J + a] + ny * geo[G_J + 2 + a];
                        double P = geo[G_J + 2 * cc + a] - nc_ * nJ;
                        acc += P * R2[((f * D::NRT + i) * 2 + a) * D::NPK + j];
                    }
                    bnd += geo[G_LEN + f] / fl[f] / det * ne * acc;
                }
                val = (vol - bnd) * sc[i];
            } else {
                int h = col - D::NRT, f = h / D::NF, m = h % D::NF;
                double ne = geo[G_NK + 2 * f + e];
                double tc = geo[G_TF + 2 * f + cc];
                double om = (m & 1) ? geo[G_O + f] : 1.0;
                val = ne * tc * sqrt(geo[G_LEN + f]) * om * R3[(f * D::NPK + j) * D::NF + m];
            }
            C[idx] = val;
        }
        for (int idx = tid; idx < D::NRT * D::NPK; idx += nt) {
            int i = idx / D::NPK;
            Dm[idx] = sgn * R5[idx] * sc[i];
        }
        for (int i = tid; i < D::NRT; i += nt) {
            double s = 0.0;
            if (forcing) {
                for (int n = 0; n < D::NLAT; ++n)
                    for (int a = 0; a < 2; ++a) {
                        double JtF = geo[G_J + a] * Fn[2 * n] + geo[G_J + 2 + a] * Fn[2 * n + 1];
                        s += JtF * R6[(i * 2 + a) * D::NLAT + n];
                    }
            }
            Fl[i] = sgn * s * sc[i];
        }
        for (int i = D::NRT + tid; i < D::NCOL; i += nt) Fl[i] = 0.0;
        __syncthreads();
        // K = (nu/|det|) CᵀC + beta M_u
        {
            double JtJ[4];
            JtJ[0] = geo[G_J + 0] * geo[G_J + 0] + geo[G_J + 2] * geo[G_J + 2];
            JtJ[1] = geo[G_J + 0] * geo[G_J + 1] + geo[G_J + 2] * geo[G_J + 3];
            JtJ[2] = JtJ[1];
            JtJ[3] = geo[G_J + 1] * geo[G_J + 1] + geo[G_J + 3] * geo[G_J + 3];
            for (int idx = tid; idx < D::NCOL * D::NCOL; idx += nt) {
                int p = idx / D::NCOL, q = idx % D::NCOL;
                double s = 0.0;
                for (int r = 0; r < D::NL; ++r) s += C[r * D::NCOL + p] * C[r * D::NCOL + q];
                s *= nu / adet;
                if (p < D::NRT && q < D::NRT && beta != 0.0) {
                    double m = 0.0;
                    for (int a = 0; a < 2; ++a)
                        for (int b = 0; b < 2; ++b)
                            m += JtJ[2 * a + b] * R4[((p * 2 + a) * D::NRT + q) * 2 + b];
                    s += beta / adet * m * sc[p] * sc[q];
                }
                Km[idx] = s;
            }
        }
        __syncthreads();
        if (conv) convection_block<K>(c, conv, conv_t, newton_x, cell_int, T, geo, sc, Km, Fl, sm);
        // global column of output unknown o: facet f, t = normal/tangential, m
        auto gcol = [&](int o) {
            int f = o / (2 * D::NF), t = (o / D::NF) & 1, m = o % D::NF;
            return t == 0 ? f * D::NF + m : D::NRT + f * D::NF + m;
        };
        if constexpr (D::NRI > 0) {
            for (int idx = tid; idx < D::NRI * D::NRI; idx += nt) {
                int r = idx / D::NRI, s = idx % D::NRI;
                Lii[idx] = Km[(3 * D::NF + r) * D::NCOL + 3 * D::NF + s];
            }
            for (int idx = tid; idx < D::NRI * D::NY; idx += nt) {
                int r = idx / D::NY, col = idx % D::NY;
                double v;
                if (col < D::NG) v = Km[(3 * D::NF + r) * D::NCOL + gcol(col)];
                else if (col < D::NG + D::NPO) v = Dm[(3 * D::NF + r) * D::NPK + (col - D::NG + 1)];
                else v = Fl[3 * D::NF + r];
                Y[idx] = v;
            }
            __syncthreads();
            if (tid == 0 && !(conv ? lu_serial(Lii, D::NRI, D::NRI, s_perm) : chol_serial(Lii, D::NRI, D::NRI)))
                s_ok = 0;
            __syncthreads();
            for (int col = tid; col < D::NY; col += nt) {
                if (conv) lu_solve_col(Lii, D::NRI, D::NRI, s_perm, Y, D::NY, col);
                else chol_solve_col(Lii, D::NRI, D::NRI, Y, D::NY, col);
            }
            __syncthreads();
            // S_p, W, v
            for (int idx = tid; idx < D::NPO * D::NPO; idx += nt) {
                int j = idx / D::NPO, j2 = idx % D::NPO;
                double s = 0.0;
                for (int r = 0; r < D::NRI; ++r)
                    s += Dm[(3 * D::NF + r) * D::NPK + j + 1] * Y[r * D::NY + D::NG + j2];
                Sp[idx] = s;
            }
            for (int idx = tid; idx < D::NPO * (D::NG + 1); idx += nt) {
                int j = idx / (D::NG + 1), col = idx % (D::NG + 1);
                double s = 0.0;
                int ycol = col < D::NG ? col : D::NG + D::NPO;
                for (int r = 0; r < D::NRI; ++r)
                    s += Dm[(3 * D::NF + r) * D::NPK + j + 1] * Y[r * D::NY + ycol];
                if (col < D::NG) {
                    int gc = gcol(col);
                    if (gc < D::NRT) s -= Dm[gc * D::NPK + j + 1];
                    Wm[j * D::NG + col] = s;
                }
                Zm[j * (D::NG + 1) + col] = s;
            }
            if (conv)   // W2 = K_gi Y_D - D_ogᵀ, stored [j][p]
                for (int idx = tid; idx < D::NPO * D::NG; idx += nt) {
                    int j = idx / D::NG, p = idx % D::NG;
                    int gp = gcol(p);
                    double s = 0.0;
                    for (int r = 0; r < D::NRI; ++r) s += Km[gp * D::NCOL + 3 * D::NF + r] * Y[r * D::NY + D::NG + j];
                    if (gp < D::NRT) s -= Dm[gp * D::NPK + j + 1];
                    W2[idx] = s;
                }
            __syncthreads();
            if (tid == 0 && !(conv ? lu_serial(Sp, D::NPO, D::NPO, s_perm) : chol_serial(Sp, D::NPO, D::NPO)))
                s_ok = 0;
            __syncthreads();
            for (int col = tid; col < D::NG + 1; col += nt) {
                if (conv) lu_solve_col(Sp, D::NPO, D::NPO, s_perm, Zm, D::NG + 1, col);
                else chol_solve_col(Sp, D::NPO, D::NPO, Zm, D::NG + 1, col);
            }
            __syncthreads();
        }
        if (rec.x) {
            // recovery of the local unknowns from the skeleton values x_g:
            //   p_o = S_p^{-1}(W x_g - D_oi Y_F),  u_i = Y_F - Y_g x_g + Y_D p_o,
            //   L = -(nu/|det J|) C [u; û]   (orthonormal P^k coefficients)
            for (int p = tid; p < D::NG; p += nt) {
                int f = p / (2 * D::NF);
                int j = rec.cell_int[3 * c + f];
                double v = 0.0;
                if (j >= 0) v = rec.x[(size_t)j * 2 * D::NF + p % (2 * D::NF)];
                else if (rec.xD && rec.cell_bnd[3 * c + f] >= 0)
                    v = rec.xD[(size_t)rec.cell_bnd[3 * c + f] * 2 * D::NF + p % (2 * D::NF)];
                xg[p] = v;
            }
            __syncthreads();
            for (int j = tid; j < D::NPO; j += nt) {
                double v = -Zm[j * (D::NG + 1) + D::NG];
                for (int q = 0; q < D::NG; ++q) v += Zm[j * (D::NG + 1) + q] * xg[q];
                po[j] = v;
            }
            __syncthreads();
            for (int col = tid; col < D::NCOL; col += nt) {
                double v = 0.0;
                if (col < 3 * D::NF) {
                    int f = col / D::NF, m = col % D::NF;
                    v = xg[f * 2 * D::NF + m];
                } else if (col < D::NRT) {
                    int r = col - 3 * D::NF;
                    v = Y[r * D::NY + D::NG + D::NPO];
                    for (int q = 0; q < D::NG; ++q) v -= Y[r * D::NY + q] * xg[q];
                    for (int j = 0; j < D::NPO; ++j) v += Y[r * D::NY + D::NG + j] * po[j];
                } else {
                    int h = col - D::NRT, f = h / D::NF, m = h % D::NF;
                    v = xg[f * 2 * D::NF + D::NF + m];
                }
                xf[col] = v;
            }
            __syncthreads();
            if (rec.L)
                for (int row = tid; row < D::NL; row += nt) {
                    double v = 0.0;
                    for (int col = 0; col < D::NCOL; ++col) v += C[row * D::NCOL + col] * xf[col];
                    rec.L[c * D::NL + row] = -nu / adet * v;
                }
            if (rec.rt)
                for (int i = tid; i < D::NRT; i += nt) rec.rt[c * D::NRT + i] = xf[i] * sc[i];
            if (rec.po)
                for (int j = tid; j < D::NPO; j += nt) rec.po[c * D::NPO + j] = po[j];
            if (rec.ulat)
                for (int idx = tid; idx < 2 * D::NLAT; idx += nt) {
                    int n = idx >> 1, cc = idx & 1;
                    double v = 0.0;
                    for (int i = 0; i < D::NRT; ++i)
                        for (int a = 0; a < 2; ++a)
                            v += geo[G_J + 2 * cc + a] * xf[i] * sc[i] * R7[(i * 2 + a) * D::NLAT + n];
                    rec.ulat[c * 2 * D::NLAT + idx] = v / det;
                }
        }
        // A = K_gg − K_gi Y_g + Wᵀ Z_W (+ AL),  F = F_g − K_gi Y_F + Wᵀ Z_v
        const double al = eps_inv / geo[G_AREA];
        const double *Wl = conv ? W2 : Wm;     // [j][p]: Wᵀ (symmetric K) or W2
        if (Aout)
        for (int idx = tid; idx < D::NG * D::NG; idx += nt) {
            // stored by row blocks: idx = (lf * NG + q) * DPF + d for row p = lf * DPF + d
            constexpr int DPF = 2 * D::NF;
            const int lfp = idx / (D::NG * DPF), rem = idx - lfp * D::NG * DPF;
            const int q = rem / DPF, p = lfp * DPF + (rem - (rem / DPF) * DPF);
            int gp = gcol(p), gq = gcol(q);
            double s = Km[gp * D::NCOL + gq];
            for (int r = 0; r < D::NRI; ++r) s -= Km[gp * D::NCOL + 3 * D::NF + r] * Y[r * D::NY + q];
            for (int j = 0; j < D::NPO; ++j) s += Wl[j * D::NG + p] * Zm[j * (D::NG + 1) + q];
            int fp = p / (2 * D::NF), fq = q / (2 * D::NF);
            if (p % (2 * D::NF) == 0 && q % (2 * D::NF) == 0)
                s += al * geo[G_SIG + fp] * sqrt(geo[G_LEN + fp]) * geo[G_SIG + fq] * sqrt(geo[G_LEN + fq]);
            Aout[c * D::NG * D::NG + idx] = s;
            if (Afout) Afout[c * D::NG * D::NG + idx] = (float)s;
        }
        if (Fout)
            for (int p = tid; p < D::NG; p += nt) {
                int gp = gcol(p);
                double s = Fl[gp];
                for (int r = 0; r < D::NRI; ++r)
                    s -= Km[gp * D::NCOL + 3 * D::NF + r] * Y[r * D::NY + D::NG + D::NPO];
                for (int j = 0; j < D::NPO; ++j) s += Wl[j * D::NG + p] * Zm[j * (D::NG + 1) + D::NG];
                Fout[c * D::NG + p] = s;
            }
        __syncthreads();
        if (tid == 0 && !s_ok) atomicOr(flag, 1);
        __syncthreads();
    }
}

template <int K>
cudaError_t launch_condense_k(const DevLevel &L, const double *ref, const RefTables &rt, double nu,
                              const double *nu_cell, double beta, double gamma, const double *forcing,
                              const double *conv, int conv_t, const double *newton_x, double *A, float *Af,
                              double *Fel, int *flag, const RecoverArgs &rec, cudaStream_t s) {
    using D = Dims<K>;
    if (conv && (rt.nq != D::NQ || rt.nfq != D::NFQ)) return cudaErrorInvalidValue;
    if (newton_x && !conv) return cudaErrorInvalidValue;
    size_t smem = sizeof(double) * (newton_x ? D::TOTAL_NEWTON : conv ? D::TOTAL_CONV : D::TOTAL);
    auto kern = condense_kernel<K>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(double) * D::TOTAL_NEWTON));
    if (e != cudaSuccess) return e;
    RefPtrs T;
    for (int i = 0; i < N_REF_TABLES; ++i) T.R[i] = ref + ref_table_offset(rt, i);
    int64_t grid = L.nc < 152 * 64 ? L.nc : 152 * 64;
    if (grid < 1) return cudaSuccess;
    note_launches(1);
    kern<<<(unsigned)grid, 128, smem, s>>>(L.nc, L.coords.p, L.cells.p, T, nu, nu_cell, beta, gamma, forcing,
                                           conv, conv_t, newton_x, L.cell_int.p, A, Af, Fel, flag, rec);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ patch inverses
// Patch matrix A_ss assembled from the cells of the vertex star (slots = patch
// facets), then inverted by Gauss-Jordan with partial pivoting (A_ss is SPD for
// Stokes and has a positive definite symmetric part for Oseen; a Newton-step
// operator need not).
__global__ void patch_inverse_kernel(int n_patches, int pf_max, int pc_max, int dpf, int nloc,
                                     int np_max, const int *__restrict__ patch_nf,
                                     const int *__restrict__ patch_nc,
                                     const int *__restrict__ patch_cells,
                                     const int *__restrict__ slot_src, const double *__restrict__ A,
                                     double *__restrict__ Pinv, float *__restrict__ Pinvf,
                                     int pivot, int *flag) {
    extern __shared__ double sm[];
    int p = blockIdx.x;
    if (p >= n_patches) return;
    int nf = patch_nf[p], ncell = patch_nc[p];
    int np = nf * dpf;
    double *M = sm;                           // np_max*np_max
    double *colp = M + np_max * np_max;       // np_max
    double *rowp = colp + np_max;             // np_max
    int *lfmap = (int *)(rowp + np_max);      // pc_max*pf_max: local facet of slot j in star cell si
    int *ipiv = lfmap + pc_max * pf_max;      // np_max: row interchanged at each step
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int i = tid; i < pc_max * pf_max; i += nt) lfmap[i] = -1;
    __syncthreads();
    if (tid == 0)
        for (int j = 0; j < nf; ++j)
            for (int q = 0; q < 2; ++q) {
                int src = slot_src[((size_t)p * pf_max + j) * 2 + q];
                lfmap[(src >> 2) * pf_max + j] = src & 3;
            }
    __syncthreads();
    for (int idx = tid; idx < np * np; idx += nt) {
        int P = idx / np, Q = idx % np;
        int j1 = P / dpf, d1 = P % dpf, j2 = Q / dpf, d2 = Q % dpf;
        double s = 0.0;
        for (int si = 0; si < ncell; ++si) {
            int l1 = lfmap[si * pf_max + j1], l2 = lfmap[si * pf_max + j2];
            if (l1 < 0 || l2 < 0) continue;
            int c = patch_cells[(size_t)p * pc_max + si];
            s += A[(size_t)c * nloc * nloc + l1 * nloc * dpf + (l2 * dpf + d2) * dpf + d1];
        }
        M[P * np + Q] = s;
    }
    __syncthreads();
    // in-place Gauss-Jordan; with `pivot` partial pivoting (the row interchanges are undone on
    // the columns of the result at the end), without it the SPD pivots are checked positive
    __shared__ int ok;
    if (tid == 0) ok = 1;
    for (int piv = 0; piv < np; ++piv) {
        __syncthreads();
        if (tid == 0) {
            int best = piv;
            double bv = fabs(M[piv * np + piv]);
            if (pivot) {
                for (int i = piv + 1; i < np; ++i)
                    if (fabs(M[i * np + piv]) > bv) {
                        bv = fabs(M[i * np + piv]);
                        best = i;
                    }
                if (!(bv > 1e-300) || !isfinite(bv)) ok = 0;
            } else if (!(M[piv * np + piv] > 0.0)) {
                ok = 0;
            }
            ipiv[piv] = best;
        }
        __syncthreads();
        const int best = ipiv[piv];
        if (best != piv)
            for (int j = tid; j < np; j += nt) {
                const double t = M[piv * np + j];
                M[piv * np + j] = M[best * np + j];
                M[best * np + j] = t;
            }
        __syncthreads();
        double d = M[piv * np + piv];
        if (!(fabs(d) > 1e-300) || !isfinite(d)) d = 1.0;
        // one reciprocal per pivot (FP64 division is a long instruction sequence; the
        // update below is then one FMA per entry)
        const double dinv = 1.0 / d;
        for (int i = tid; i < np; i += nt) {
            colp[i] = M[i * np + piv];
            rowp[i] = M[piv * np + i] * dinv;
        }
        __syncthreads();
        // warp w updates rows w, w + nwarps, ...; its lanes walk the columns
        for (int i = tid >> 5; i < np; i += nt >> 5) {
            const double ci = colp[i];
            for (int j = tid & 31; j < np; j += 32) {
                double v;
                if (i == piv) v = (j == piv) ? dinv : rowp[j];
                else if (j == piv) v = -ci * dinv;
                else v = fma(-ci, rowp[j], M[i * np + j]);
                M[i * np + j] = v;
            }
        }
    }
    __syncthreads();
    for (int piv = np - 1; piv >= 0; --piv) {
        const int q = ipiv[piv];
        if (q != piv)
            for (int i = tid; i < np; i += nt) {
                const double t = M[i * np + piv];
                M[i * np + piv] = M[i * np + q];
                M[i * np + q] = t;
            }
        __syncthreads();
    }
    // stored transposed, Pinv[j][i] = (A_ss^{-1})_ij, for the column-reading smoother
    for (int idx = tid; idx < np_max * np_max; idx += nt) {
        int j = idx / np_max, i = idx % np_max;
        double v = (i < np && j < np) ? M[i * np + j] : 0.0;
        Pinv[(size_t)p * np_max * np_max + idx] = v;
        if (Pinvf) Pinvf[(size_t)p * np_max * np_max + idx] = (float)v;
    }
    if (tid == 0 && !ok) atomicOr(flag, 2);
}

// ------------------------------------------------------------------ harmonic extension
// Per coarse cell: A_TT, A_TB from the four children's lowest-order matrices
// (slots 6..8 = T, 0..5 = B, two unknowns per slot), H = -A_TT^{-1} A_TB.
__global__ void transfer_H_kernel(int64_t ncc, const int *__restrict__ children,
                                  const int *__restrict__ child_slot, const int *__restrict__ slots,
                                  const double *__restrict__ A0, double *__restrict__ Hout,
                                  float *__restrict__ Hf, int *flag) {
    int64_t P = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (P >= ncc) return;
    double M[18][18];
    for (int i = 0; i < 18; ++i)
        for (int j = 0; j < 18; ++j) M[i][j] = 0.0;
    for (int ch = 0; ch < 4; ++ch) {
        int c = children[4 * P + ch];
        const double *Ac = A0 + (size_t)c * 36;
        for (int l1 = 0; l1 < 3; ++l1) {
            int s1 = child_slot[12 * P + 3 * ch + l1];
            for (int l2 = 0; l2 < 3; ++l2) {
                int s2 = child_slot[12 * P + 3 * ch + l2];
                for (int a = 0; a < 2; ++a)
                    for (int b = 0; b < 2; ++b) M[2 * s1 + a][2 * s2 + b] += Ac[l1 * 12 + (2 * l2 + b) * 2 + a];
            }
        }
    }
    // LU of A_TT (rows/cols 12..17) without pivoting: SPD for Stokes, positive
    // definite symmetric part for Oseen
    double Lm[6][6];
    bool ok = true;
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) Lm[i][j] = M[12 + i][12 + j];
    for (int j = 0; j < 6; ++j) {
        double d = Lm[j][j];
        if (!(d > 0.0)) { ok = false; d = 1.0; Lm[j][j] = 1.0; }
        for (int i = j + 1; i < 6; ++i) {
            double l = Lm[i][j] / d;
            Lm[i][j] = l;
            for (int c2 = j + 1; c2 < 6; ++c2) Lm[i][c2] -= l * Lm[j][c2];
        }
    }
    for (int col = 0; col < 12; ++col) {
        int s = col / 2;
        bool has = slots[9 * P + s] >= 0;
        double x[6];
        for (int i = 0; i < 6; ++i) x[i] = has ? -M[12 + i][col] : 0.0;
        for (int i = 0; i < 6; ++i) {
            double v = x[i];
            for (int p = 0; p < i; ++p) v -= Lm[i][p] * x[p];
            x[i] = v;
        }
        for (int i = 5; i >= 0; --i) {
            double v = x[i];
            for (int p = i + 1; p < 6; ++p) v -= Lm[i][p] * x[p];
            x[i] = v / Lm[i][i];
        }
        for (int i = 0; i < 6; ++i) {
            Hout[72 * P + i * 12 + col] = x[i];
            Hf[72 * P + i * 12 + col] = (float)x[i];
        }
    }
    if (!ok) atomicOr(flag, 4);
}

// ------------------------------------------------------------------ coarse dense inverse
__global__ void coarse_assemble_kernel(int64_t n_int, int dim, const int *__restrict__ facet_adj,
                                       const int *__restrict__ cell_int, const double *__restrict__ A0,
                                       double *__restrict__ M, int64_t n) {
    int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (row >= n) return;
    // lowest order: dim unknowns per facet, dim+1 facets per cell, element matrices nloc x nloc
    const int nfc = dim + 1, nloc = nfc * dim;
    int64_t i = row / dim;
    int d = row % dim;
    double *Mr = M + row * n;
    for (int64_t j = 0; j < n; ++j) Mr[j] = 0.0;
    for (int q = 0; q < 2; ++q) {
        int adj = facet_adj[2 * i + q];
        if (adj < 0) continue;
        int c = adj >> 2, lf = adj & 3;
        for (int col = 0; col < nloc; ++col) {
            int jf = cell_int[nfc * c + col / dim];
            if (jf < 0) continue;
            Mr[dim * jf + col % dim] += A0[(size_t)c * nloc * nloc + lf * nloc * dim + col * dim + d];
        }
    }
}

// Gauss-Jordan step at pivot piv (SPD coarsest matrix, no pivoting): save the pivot column and
// the pivot row divided by the pivot (and the pivot's reciprocal at rowp[n]), so that the update
// is one FMA per entry
__global__ void gj_save_kernel(const double *M, int64_t n, int64_t piv, double *colp, double *rowp,
                               int *flag) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double d = M[piv * n + piv];
    if (!(d > 0.0)) d = 1.0;
    const double dinv = 1.0 / d;
    if (i < n) {
        colp[i] = M[i * n + piv];
        rowp[i] = M[piv * n + i] * dinv;
    }
    if (i == 0) {
        rowp[n] = dinv;
        if (!(M[piv * n + piv] > 0.0)) atomicOr(flag, 8);
    }
}

// one row per blockIdx.y, columns across x: no integer division per entry
__global__ void gj_update_kernel(double *M, int64_t n, int64_t piv, const double *colp,
                                 const double *rowp) {
    const int64_t i = blockIdx.y;
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    const double dinv = rowp[n], ci = colp[i];
    double *Mi = M + i * n;
    double v;
    if (i == piv) v = j == piv ? dinv : rowp[j];
    else if (j == piv) v = -ci * dinv;
    else v = fma(-ci, rowp[j], Mi[j]);
    Mi[j] = v;
}

// ------------------------------------------------------------------ geometry, loads
__global__ void cell_geometry_kernel(int64_t nc, const double *coords, const int *cells,
                                     double *cell_d, double *cell_area) {
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= nc) return;
    double geo[64];
    cell_geometry(coords, cells, c, geo);
    for (int f = 0; f < 3; ++f) cell_d[3 * c + f] = geo[G_SIG + f] * sqrt(geo[G_LEN + f]);
    cell_area[c] = geo[G_AREA];
}

__global__ void assemble_load_kernel(int64_t n_int, int dpf, int nfc, const int *__restrict__ facet_adj,
                                     const double *__restrict__ Fel, double *__restrict__ F) {
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n_int * dpf) return;
    int64_t i = idx / dpf;
    int d = idx % dpf;
    double s = 0.0;
    for (int q = 0; q < 2; ++q) {
        int adj = facet_adj[2 * i + q];
        if (adj < 0) continue;
        int c = adj >> 2, lf = adj & 3;
        s += Fel[(size_t)c * nfc * dpf + lf * dpf + d];
    }
    F[idx] = s;
}

unsigned blocks_for(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// ------------------------------------------------------------------ convecting field per level
// Lowest-order levels carry the RT_0 field whose facet fluxes are those of the
// finest field (mean of the two sides), summed over the two fine halves of
// every coarse facet; it is handed to the condensation as values at the cell
// vertices (the degree-1 lattice).

// outward flux ∫_{F_f} w·n_K of the lattice field through each local facet
__global__ void conv_flux_kernel(int64_t nc, const double *__restrict__ coords, const int *__restrict__ cells,
                                 int nlat, int nfq, const double *__restrict__ R14, const double *__restrict__ R16,
                                 const double *__restrict__ conv, double *__restrict__ flux) {
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= nc) return;
    double geo[64];
    cell_geometry(coords, cells, c, geo);
    const double *w = conv + c * 2 * nlat;
    for (int f = 0; f < 3; ++f) {
        double s = 0.0;
        for (int g = 0; g < nfq; ++g) {
            double wx = 0.0, wy = 0.0;
            for (int n = 0; n < nlat; ++n) {
                const double l = R14[(f * nfq + g) * nlat + n];
                wx += l * w[2 * n];
                wy += l * w[2 * n + 1];
            }
            s += R16[g] * (wx * geo[G_NK + 2 * f] + wy * geo[G_NK + 2 * f + 1]);
        }
        flux[3 * c + f] = geo[G_LEN + f] * s;
    }
}

// both sides of an interior facet take the mean of their (opposite) fluxes
__global__ void flux_consistent_kernel(int64_t n_int, const int *__restrict__ facet_adj, double *__restrict__ flux) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_int) return;
    const int a0 = facet_adj[2 * i], a1 = facet_adj[2 * i + 1];
    if (a0 < 0 || a1 < 0) return;
    const int64_t e0 = 3 * (int64_t)(a0 >> 2) + (a0 & 3), e1 = 3 * (int64_t)(a1 >> 2) + (a1 & 3);
    const double v = 0.5 * (flux[e0] - flux[e1]);
    flux[e0] = v;
    flux[e1] = -v;
}

// coarse outward flux through local facet f = sum over the fine facets in slots 2f, 2f+1
__global__ void flux_restrict_kernel(int64_t ncc, const int *__restrict__ children,
                                     const int *__restrict__ child_slot, const double *__restrict__ ff,
                                     double *__restrict__ fc) {
    int64_t P = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (P >= ncc) return;
    double s[3] = {0.0, 0.0, 0.0};
    for (int ch = 0; ch < 4; ++ch) {
        const int64_t c = children[4 * P + ch];
        for (int lf = 0; lf < 3; ++lf) {
            const int slot = child_slot[12 * P + 3 * ch + lf];
            if (slot >= 0 && slot < 6) s[slot / 2] += ff[3 * c + lf];
        }
    }
    for (int f = 0; f < 3; ++f) fc[3 * P + f] = s[f];
}

// RT_0 field with outward fluxes Φ_f at the vertices: w(X_v) = Σ_{f≠v} Φ_f (X_v − X_f) / (2|K|)
__global__ void rt0_vertex_kernel(int64_t nc, const double *__restrict__ coords, const int *__restrict__ cells,
                                  const double *__restrict__ flux, double *__restrict__ out) {
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= nc) return;
    double X[3][2];
    for (int i = 0; i < 3; ++i) {
        const int v = cells[3 * c + i];
        X[i][0] = coords[2 * v];
        X[i][1] = coords[2 * v + 1];
    }
    const double det = (X[1][0] - X[0][0]) * (X[2][1] - X[0][1]) - (X[2][0] - X[0][0]) * (X[1][1] - X[0][1]);
    const double two_area = fabs(det);
    for (int v = 0; v < 3; ++v)
        for (int d = 0; d < 2; ++d) {
            double s = 0.0;
            for (int f = 0; f < 3; ++f)
                if (f != v) s += flux[3 * c + f] * (X[v][d] - X[f][d]);
            out[6 * c + 2 * v + d] = s / two_area;
        }
}

// row-major copies of the stored element matrices: out[b][p][q] = A_pq, stored at
// in[b][(p / dpf) * n * dpf + q * dpf + p % dpf]
__global__ void unpack_blocks_kernel(int64_t nblk, int n, int dpf, const double *__restrict__ in,
                                     double *__restrict__ out) {
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nn = (int64_t)n * n;
    if (idx >= nblk * nn) return;
    const int64_t b = idx / nn;
    const int r = (int)(idx - b * nn), p = r / n, q = r % n;
    out[idx] = in[b * nn + (int64_t)(p / dpf) * n * dpf + (int64_t)q * dpf + p % dpf];
}

// coarse-cell viscosity = mean over its four children (equal areas under red refinement)
__global__ void nu_average_kernel(int64_t ncc, const int *__restrict__ children, const double *__restrict__ nu_f,
                                  double *__restrict__ nu_c) {
    int64_t P = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (P >= ncc) return;
    double s = 0.0;
    for (int ch = 0; ch < 4; ++ch) s += nu_f[children[4 * P + ch]];
    nu_c[P] = 0.25 * s;
}

// Adjoint gradients (Stokes: the transposed local system equals the primal one with the
// signs of the flux and pressure blocks flipped, so lambda_L = -L^a, lambda_u = u^a):
//   dJ/dnu_K = -nu_K^{-2} (L_h, L^a)_K = -nu_K^{-2} |det J| sum_r L_r L^a_r   (orthonormal P^k)
//   dJ/dF_{K,n,c} = (u^a, lam_n e_c)_K = sgn(det J) sum_i rt^a_i sum_a J[c][a] R6[i][a][n]
template <int K>
__global__ void adjoint_gradient_kernel(int64_t nc, const double *__restrict__ coords, const int *__restrict__ cells,
                                        const double *__restrict__ R6, double nu_scalar,
                                        const double *__restrict__ nu_cell, const double *__restrict__ Lp,
                                        const double *__restrict__ La, const double *__restrict__ rta,
                                        double *__restrict__ grad_nu, double *__restrict__ grad_f) {
    using D = Dims<K>;
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= nc) return;
    double geo[64];
    cell_geometry(coords, cells, c, geo);
    const double nu = nu_cell ? nu_cell[c] : nu_scalar;
    if (grad_nu) {
        double s = 0.0;
        for (int r = 0; r < D::NL; ++r) s += Lp[c * D::NL + r] * La[c * D::NL + r];
        grad_nu[c] = -fabs(geo[G_DET]) * s / (nu * nu);
    }
    if (grad_f)
        for (int n = 0; n < D::NLAT; ++n)
            for (int cc = 0; cc < 2; ++cc) {
                double v = 0.0;
                for (int i = 0; i < D::NRT; ++i)
                    for (int a = 0; a < 2; ++a) v += rta[c * D::NRT + i] * geo[G_J + 2 * cc + a] * R6[(i * 2 + a) * D::NLAT + n];
                grad_f[(c * D::NLAT + n) * 2 + cc] = geo[G_SGN] * v;
            }
}

// per-cell 0.5 ||u_h - u_target||^2_K for lattice samples of two [P^{k+1}]^2 fields, and e = u_h - u_t
template <int K>
__global__ void objective_kernel(int64_t nc, const double *__restrict__ coords, const int *__restrict__ cells,
                                 const double *__restrict__ R8, const double *__restrict__ ulat,
                                 const double *__restrict__ utgt, double *__restrict__ e_out,
                                 double *__restrict__ jcell) {
    using D = Dims<K>;
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= nc) return;
    double geo[64];
    cell_geometry(coords, cells, c, geo);
    double e[2 * D::NLAT];
    for (int i = 0; i < 2 * D::NLAT; ++i) {
        e[i] = ulat[c * 2 * D::NLAT + i] - utgt[c * 2 * D::NLAT + i];
        e_out[c * 2 * D::NLAT + i] = e[i];
    }
    double s = 0.0;
    for (int n = 0; n < D::NLAT; ++n)
        for (int m = 0; m < D::NLAT; ++m)
            s += R8[n * D::NLAT + m] * (e[2 * n] * e[2 * m] + e[2 * n + 1] * e[2 * m + 1]);
    jcell[c] = 0.5 * fabs(geo[G_DET]) * s;
}

} // namespace

cudaError_t launch_nu_average(const DevLevel &fine, const double *nu_f, double *nu_c, cudaStream_t s) {
    if (fine.nc_coarse == 0) return cudaSuccess;
    note_launches(1);
    nu_average_kernel<<<blocks_for(fine.nc_coarse, 128), 128, 0, s>>>(fine.nc_coarse, fine.tr_children.p, nu_f, nu_c);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_gradient(int k, const DevLevel &L, const double *ref, const RefTables &rt,
                                    double nu, const double *nu_cell, const double *Lp, const double *La,
                                    const double *rta, double *grad_nu, double *grad_f, cudaStream_t s) {
    const double *R6 = ref + ref_table_offset(rt, 5);
    unsigned nb = blocks_for(L.nc, 64);
    note_launches(1);
    switch (k) {
    case 0: adjoint_gradient_kernel<0><<<nb, 64, 0, s>>>(L.nc, L.coords.p, L.cells.p, R6, nu, nu_cell, Lp, La, rta, grad_nu, grad_f); break;
    case 1: adjoint_gradient_kernel<1><<<nb, 64, 0, s>>>(L.nc, L.coords.p, L.cells.p, R6, nu, nu_cell, Lp, La, rta, grad_nu, grad_f); break;
    case 2: adjoint_gradient_kernel<2><<<nb, 64, 0, s>>>(L.nc, L.coords.p, L.cells.p, R6, nu, nu_cell, Lp, La, rta, grad_nu, grad_f); break;
    case 3: adjoint_gradient_kernel<3><<<nb, 64, 0, s>>>(L.nc, L.coords.p, L.cells.p, R6, nu, nu_cell, Lp, La, rta, grad_nu, grad_f); break;
    case 4: adjoint_gradient_kernel<4><<<nb, 64, 0, s>>>(L.nc, L.coords.p, L.cells.p, R6, nu, nu_cell, Lp, La, rta, grad_nu, grad_f); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_objective(int k, const DevLevel &L, const double *ref, const RefTables &rt, const double *ulat,
                             const double *utgt, double *e_out, double *jcell, cudaStream_t s) {
    const double *R8 = ref + ref_table_offset(rt, 7);
    unsigned nb = blocks_for(L.nc, 64);
    note_launches(1);
    switch (k) {
    case 0: objective_kernel<0><<<nb, 64, 0, s>>>(L.nc, L.coords.p, L.cells.p, R8, ulat, utgt, e_out, jcell); break;
    case 1: objective_kernel<1><<<nb, 64, 0, s>>>(L.nc, L.coords.p, L.cells.p, R8, ulat, utgt, e_out, jcell); break;
    case 2: objective_kernel<2><<<nb, 64, 0, s>>>(L.nc, L.coords.p, L.cells.p, R8, ulat, utgt, e_out, jcell); break;
    case 3: objective_kernel<3><<<nb, 64, 0, s>>>(L.nc, L.coords.p, L.cells.p, R8, ulat, utgt, e_out, jcell); break;
    case 4: objective_kernel<4><<<nb, 64, 0, s>>>(L.nc, L.coords.p, L.cells.p, R8, ulat, utgt, e_out, jcell); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_condense(int k, const DevLevel &L, const double *ref, const RefTables &rt, double nu,
                            const double *nu_cell, double beta, double gamma, const double *forcing,
                            const double *conv, int conv_t, const double *newton_x, double *A, float *Af,
                            double *Fel, int *flag, const RecoverArgs &rec, cudaStream_t s) {
    switch (k) {
#define HDG_CONDENSE_CASE(KK)                                                                         \
    case KK:                                                                                          \
        return launch_condense_k<KK>(L, ref, rt, nu, nu_cell, beta, gamma, forcing, conv, conv_t, newton_x, \
                                     A, Af, Fel, flag, rec, s);
        HDG_CONDENSE_CASE(0)
        HDG_CONDENSE_CASE(1)
        HDG_CONDENSE_CASE(2)
        HDG_CONDENSE_CASE(3)
        HDG_CONDENSE_CASE(4)
#undef HDG_CONDENSE_CASE
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_patch_inverse(const DevLevel &L, const DevOperator &op, int pivot, int *flag, cudaStream_t s) {
    if (L.n_patches == 0) return cudaSuccess;
    size_t smem = sizeof(double) * ((size_t)op.np_max * op.np_max + 2 * op.np_max) +
                  sizeof(int) * ((size_t)L.pc_max * L.pf_max + op.np_max);
    cudaError_t e = cudaFuncSetAttribute(patch_inverse_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    note_launches(1);
    patch_inverse_kernel<<<L.n_patches, 256, smem, s>>>(
        L.n_patches, L.pf_max, L.pc_max, op.dpf, op.nloc, op.np_max, L.patch_nf.p, L.patch_nc.p,
        L.patch_cells.p, L.patch_slot_src.p, op.A.p, op.Pinv.p, op.Pinvf.p, pivot, flag);
    return cudaGetLastError();
}

cudaError_t launch_transfer_H(const DevLevel &F, int *flag, cudaStream_t s) {
    if (F.nc_coarse == 0) return cudaSuccess;
    note_launches(1);
    transfer_H_kernel<<<blocks_for(F.nc_coarse, 64), 64, 0, s>>>(
        F.nc_coarse, F.tr_children.p, F.tr_child_slot.p, F.tr_slots.p, F.op0.A.p, F.tr_H.p,
        F.tr_Hf.p, flag);
    return cudaGetLastError();
}

cudaError_t launch_coarse_inverse(const DevLevel &L0, double *inv, int64_t n, int *flag,
                                  cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    note_launches(1);
    coarse_assemble_kernel<<<blocks_for(n, 128), 128, 0, s>>>(L0.n_int, L0.dim, L0.facet_adj.p, L0.cell_int.p,
                                                              L0.op0.A.p, inv, n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    double *tmp = nullptr;
    e = cudaMallocAsync(&tmp, sizeof(double) * (2 * n + 1), s);
    if (e != cudaSuccess) return e;
    const dim3 ugrid(blocks_for(n, 256), (unsigned)n);
    for (int64_t piv = 0; piv < n; ++piv) {
        note_launches(1);
        gj_save_kernel<<<blocks_for(n, 256), 256, 0, s>>>(inv, n, piv, tmp, tmp + n, flag);
        note_launches(1);
        gj_update_kernel<<<ugrid, 256, 0, s>>>(inv, n, piv, tmp, tmp + n);
    }
    e = cudaGetLastError();
    cudaFreeAsync(tmp, s);
    return e;
}

cudaError_t launch_cell_geometry(DevLevel &L, cudaStream_t s) {
    if (L.nc == 0) return cudaSuccess;
    note_launches(1);
    cell_geometry_kernel<<<blocks_for(L.nc, 128), 128, 0, s>>>(L.nc, L.coords.p, L.cells.p,
                                                               L.cell_d.p, L.cell_area.p);
    return cudaGetLastError();
}

cudaError_t launch_assemble_load(const DevLevel &L, const DevOperator &op, double *F, cudaStream_t s) {
    int64_t n = L.n_int * op.dpf;
    if (n == 0) return cudaSuccess;
    note_launches(1);
    assemble_load_kernel<<<blocks_for(n, 256), 256, 0, s>>>(L.n_int, op.dpf, L.dim + 1, L.facet_adj.p, op.Fel.p, F);
    return cudaGetLastError();
}

cudaError_t launch_conv_flux(const DevLevel &L, const double *ref, const RefTables &rt, const double *conv,
                             double *flux, cudaStream_t s) {
    if (L.nc == 0) return cudaSuccess;
    note_launches(L.n_int > 0 ? 2 : 1);
    conv_flux_kernel<<<blocks_for(L.nc, 128), 128, 0, s>>>(L.nc, L.coords.p, L.cells.p, rt.nlat, rt.nfq,
                                                           ref + ref_table_offset(rt, 13),
                                                           ref + ref_table_offset(rt, 15), conv, flux);
    if (L.n_int > 0) flux_consistent_kernel<<<blocks_for(L.n_int, 256), 256, 0, s>>>(L.n_int, L.facet_adj.p, flux);
    return cudaGetLastError();
}

cudaError_t launch_flux_restrict(const DevLevel &fine, const double *ff, double *fc, cudaStream_t s) {
    if (fine.nc_coarse == 0) return cudaSuccess;
    note_launches(1);
    flux_restrict_kernel<<<blocks_for(fine.nc_coarse, 128), 128, 0, s>>>(fine.nc_coarse, fine.tr_children.p,
                                                                         fine.tr_child_slot.p, ff, fc);
    return cudaGetLastError();
}

cudaError_t launch_rt0_vertex(const DevLevel &L, const double *flux, double *out, cudaStream_t s) {
    if (L.nc == 0) return cudaSuccess;
    note_launches(1);
    rt0_vertex_kernel<<<blocks_for(L.nc, 128), 128, 0, s>>>(L.nc, L.coords.p, L.cells.p, flux, out);
    return cudaGetLastError();
}

cudaError_t launch_unpack_blocks(int64_t nblk, int n, int dpf, const double *in, double *out, cudaStream_t s) {
    const int64_t total = nblk * (int64_t)n * n;
    if (total == 0) return cudaSuccess;
    note_launches(1);
    unpack_blocks_kernel<<<blocks_for(total, 256), 256, 0, s>>>(nblk, n, dpf, in, out);
    return cudaGetLastError();
}

} // namespace hdg
