// Static condensation on tetrahedra (Section 3.2, eq. stWeak with d = 3), FP64.
//
// One thread block per cell (grid-stride).  With the reference tables of reference3d.cpp
// and the cell's affine map x = X0 + J x^ (u = J u^ / |det J|, which keeps outward fluxes):
//  1. geometry: J, J^-1, and per face the sorted global vertex order (which fixes the face
//     frame t1, t2, n_F and basis), its area, the outward normal n_K and sigma = n_F . n_K;
//  2. the flux variable L is eliminated in closed form: its mass matrix is |det J|/nu times the
//     identity in the orthonormal basis g_j, so it adds (nu/|det J|) B^T B to the (u, û) block,
//     B being the rows (d_e u_c, g_j) - <tng(u)_c n_e, g_j> + <û_c n_e, g_j> of eq. stWeak;
//  3. beta (u, v), the pressure coupling -(p, div v) / (div u, q) and the load (f, v) are added,
//     and the interior RT moments and the mean-free pressure are eliminated by Gaussian
//     elimination in that order (the interior velocity block is SPD, and after it the pressure
//     block is R5 K^-1 R5^T > 0, so no pivoting is needed);
//  4. the face normal-moment unknowns are rotated from the reference face basis to the
//     global one, T_f = sigma |F|^(1/2) Q_p (Q_p: the face-order transform of the face's
//     sorted vertex order p), the tangential ones are already in the global frame; the
//     augmented-Lagrangian term eps^-1 |K|^-1 d d^T (d = the faces' sigma |F|^(1/2) on the
//     constant normal moment) is added.
// Outputs: element matrices A [nc][nloc][nloc] in the facet-row-block layout of the apply
// and sweep kernels (row (lf, d), column col at lf*nloc*dpf + col*dpf + d), optional FP32
// copies, element loads Fel [nc][nloc], flux weights cell_d [nc][4] and volumes cell_area.
#include "hdg3d_internal.h"

namespace hdg {
namespace {

unsigned blocks_for(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

__constant__ int FV3D[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};

template <int K>
struct Dims3 {
    static constexpr int NPK = (K + 1) * (K + 2) * (K + 3) / 6;
    static constexpr int NF = (K + 1) * (K + 2) / 2;
    static constexpr int NRT = (K + 1) * (K + 2) * (K + 4) / 2;
    static constexpr int NLAT = (K + 2) * (K + 3) * (K + 4) / 6;
    static constexpr int NUH = NRT + 8 * NF;
    static constexpr int N = NUH + NPK;
    static constexpr int NRHS = 3 * NLAT;
    static constexpr int LD = N + NRHS;
    static constexpr int DPF = 3 * NF;
    static constexpr int NLOC = 4 * DPF;
    static constexpr int NB = 9 * NPK * NUH;          // doubles of B
    static constexpr int NR = NLOC * (NLOC + NRHS);   // doubles of the row-rotated global block
    static constexpr int SCR = NB + N * LD + NR;      // doubles of scratch per block
};

template <int K>
__global__ void __launch_bounds__(128)
condense3_kernel(int64_t nc, const double *__restrict__ coords, const int *__restrict__ cells,
                 const double *__restrict__ ref, double nu, const double *__restrict__ nu_cell, double beta,
                 double gamma, const double *__restrict__ forcing, double *__restrict__ Aout,
                 float *__restrict__ Af, double *__restrict__ Fel, double *__restrict__ cell_d,
                 double *__restrict__ cell_area, double *__restrict__ scratch, int *flag, Recover3 rec) {
    using D = Dims3<K>;
    constexpr int NPK = D::NPK, NF = D::NF, NRT = D::NRT, NLAT = D::NLAT, NUH = D::NUH, N = D::N,
                  LD = D::LD, DPF = D::DPF, NLOC = D::NLOC;
    const double *R1 = ref;
    const double *R2 = R1 + NRT * 9 * NPK;
    const double *R3 = R2 + 4 * NRT * 3 * NPK;
    const double *R4 = R3 + 4 * NPK * NF;
    const double *R5 = R4 + NRT * 3 * NRT * 3;
    const double *R6 = R5 + NRT * NPK;
    const double *Q = R6 + NRT * 3 * NLAT;
    const double *FA = Q + 6 * NF * NF;
    const double *R7 = FA + 4;
    double *Bm = scratch + (size_t)blockIdx.x * D::SCR;   // [9 NPK][NUH]
    double *Km = Bm + D::NB;                              // [N][LD]
    double *Rm = Km + (size_t)N * LD;                     // [NLOC][NLOC + NRHS]
    __shared__ double J[3][3], Ji[3][3], adet, nuc;
    __shared__ double nK[4][3], t1[4][3], t2[4][3], nJ[4][3], farea[4], fsig[4];
    __shared__ int fperm[4];
    __shared__ double colq[N], rowq[LD];
    __shared__ double Xs[NUH], xl[NLOC];      // recovery: reference-basis unknowns, the cell's skeleton values
    __shared__ int bad;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int64_t c = blockIdx.x; c < nc; c += gridDim.x) {
        if (tid == 0) {
            double X[4][3];
            int gv[4];
            for (int v = 0; v < 4; ++v) {
                gv[v] = cells[4 * c + v];
                for (int d = 0; d < 3; ++d) X[v][d] = coords[3 * (size_t)gv[v] + d];
            }
            for (int r = 0; r < 3; ++r)
                for (int a = 0; a < 3; ++a) J[r][a] = X[a + 1][r] - X[0][r];
            const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                               J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                               J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
            const double id = 1.0 / det;
            Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) * id;
            Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
            Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
            Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) * id;
            Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
            Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
            Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) * id;
            Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
            Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
            adet = fabs(det);
            nuc = nu_cell ? nu_cell[c] : nu;
            bad = !(adet > 0.0) || !isfinite(adet);
            for (int f = 0; f < 4; ++f) {
                const int *cv = FV3D[f];
                // sorted global order of the canonical vertices: positions s0, s1, s2
                int s[3] = {0, 1, 2};
                for (int i = 0; i < 3; ++i)
                    for (int j = i + 1; j < 3; ++j)
                        if (gv[cv[s[j]]] < gv[cv[s[i]]]) {
                            int t = s[i];
                            s[i] = s[j];
                            s[j] = t;
                        }
                fperm[f] = s[0] == 0 ? (s[1] == 1 ? 0 : 1) : s[0] == 1 ? (s[1] == 0 ? 2 : 3) : (s[1] == 0 ? 4 : 5);
                const double *xa = X[cv[s[0]]], *xb = X[cv[s[1]]], *xc = X[cv[s[2]]];
                double e1[3], e2[3], cr[3];
                for (int d = 0; d < 3; ++d) {
                    e1[d] = xb[d] - xa[d];
                    e2[d] = xc[d] - xa[d];
                }
                cr[0] = e1[1] * e2[2] - e1[2] * e2[1];
                cr[1] = e1[2] * e2[0] - e1[0] * e2[2];
                cr[2] = e1[0] * e2[1] - e1[1] * e2[0];
                const double ncr = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
                const double ne1 = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
                double nF[3], u1[3];
                for (int d = 0; d < 3; ++d) {
                    nF[d] = cr[d] / ncr;
                    u1[d] = e1[d] / ne1;
                }
                double side = 0.0;
                for (int d = 0; d < 3; ++d) side += nF[d] * (xa[d] - X[f][d]);
                const double sg = side > 0 ? 1.0 : -1.0;
                fsig[f] = sg;
                farea[f] = 0.5 * ncr;
                t2[f][0] = nF[1] * u1[2] - nF[2] * u1[1];
                t2[f][1] = nF[2] * u1[0] - nF[0] * u1[2];
                t2[f][2] = nF[0] * u1[1] - nF[1] * u1[0];
                for (int d = 0; d < 3; ++d) {
                    nK[f][d] = sg * nF[d];
                    t1[f][d] = u1[d];
                }
                for (int a = 0; a < 3; ++a) nJ[f][a] = nK[f][0] * J[0][a] + nK[f][1] * J[1][a] + nK[f][2] * J[2][a];
                cell_d[4 * c + f] = sg * sqrt(farea[f]);
            }
            cell_area[c] = adet / 6.0;
        }
        __syncthreads();
        if (bad) {
            if (tid == 0) atomicOr(flag, 1);
            __syncthreads();
            continue;
        }
        // B: rows (c_, e, j), columns u_i (i < NRT) and û (f, a, m)
        for (int idx = tid; idx < 9 * NPK * NUH; idx += nt) {
            const int r = idx / NUH, x = idx % NUH;
            const int ce = r / NPK, j = r % NPK, cc = ce / 3, e = ce % 3;
            double v = 0.0;
            if (x < NRT) {
                const double *r1 = R1 + (size_t)x * 9 * NPK + j;
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) v += J[cc][a] * Ji[b][e] * r1[(a * 3 + b) * NPK];
                for (int f = 0; f < 4; ++f) {
                    const double s = nK[f][e] * farea[f] / (FA[f] * adet);
                    const double *r2 = R2 + ((size_t)f * NRT + x) * 3 * NPK + j;
                    double w = 0.0;
                    for (int a = 0; a < 3; ++a) w += (J[cc][a] - nK[f][cc] * nJ[f][a]) * r2[a * NPK];
                    v -= s * w;
                }
            } else {
                const int hx = x - NRT, f = hx / (2 * NF), a = (hx / NF) % 2, m = hx % NF;
                const double *q = Q + ((size_t)fperm[f] * NF + m) * NF;
                const double *r3 = R3 + ((size_t)f * NPK + j) * NF;
                double w = 0.0;
                for (int m2 = 0; m2 < NF; ++m2) w += q[m2] * r3[m2];
                v = (a == 0 ? t1[f][cc] : t2[f][cc]) * nK[f][e] * sqrt(farea[f]) / FA[f] * w;
            }
            Bm[idx] = v;
        }
        __syncthreads();
        // K = (nu/|det J|) B^T B + beta (u, v) + pressure coupling; load columns from N on
        const double sL = nuc / adet, sB = beta / adet;
        double G[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) G[a][b] = J[0][a] * J[0][b] + J[1][a] * J[1][b] + J[2][a] * J[2][b];
        for (int idx = tid; idx < N * LD; idx += nt) {
            const int x = idx / LD, y = idx % LD;
            double v = 0.0;
            if (y < NUH && x < NUH) {
                for (int r = 0; r < 9 * NPK; ++r) v += Bm[r * NUH + x] * Bm[r * NUH + y];
                v *= sL;
                if (x < NRT && y < NRT && beta != 0.0) {
                    const double *r4 = R4 + (size_t)x * 3 * NRT * 3 + y * 3;
                    double w = 0.0;
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b) w += G[a][b] * r4[a * NRT * 3 + b];
                    v += sB * w;
                }
            } else if (y < N) {
                if (x < NRT && y >= NUH) v = -R5[x * NPK + (y - NUH)];
                else if (x >= NUH && y < NRT) v = R5[y * NPK + (x - NUH)];
            } else if (x < NRT) {
                const int col = y - N, n = col / 3, cc = col % 3;
                const double *r6 = R6 + (size_t)x * 3 * NLAT + n;
                v = J[cc][0] * r6[0] + J[cc][1] * r6[NLAT] + J[cc][2] * r6[2 * NLAT];
            }
            Km[idx] = v;
        }
        __syncthreads();
        if (rec.x) {
            // recovery: the local right-hand side (f, v) - K_lg x_g in column N, with the skeleton
            // values rotated to the reference face basis (x_ref = T^T x)
            for (int l = tid; l < NLOC; l += nt) {
                const int j = rec.cell_int[4 * c + l / DPF];
                const int b = rec.xD ? rec.cell_bnd[4 * c + l / DPF] : -1;
                xl[l] = j >= 0 ? rec.x[(size_t)j * DPF + l % DPF] : b >= 0 ? rec.xD[(size_t)b * DPF + l % DPF] : 0.0;
            }
            __syncthreads();
            for (int x = tid; x < NUH; x += nt) {
                double v = 0.0;
                if (x < 4 * NF) {
                    const int f = x / NF, m2 = x % NF;
                    for (int m = 0; m < NF; ++m)
                        v += fsig[f] * sqrt(farea[f]) * Q[((size_t)fperm[f] * NF + m) * NF + m2] * xl[f * DPF + m];
                } else if (x >= NRT) {
                    const int hx = x - NRT, f = hx / (2 * NF);
                    v = xl[f * DPF + NF + hx % (2 * NF)];
                }
                Xs[x] = v;
            }
            __syncthreads();
            for (int i = tid; i < N; i += nt) {
                double v = 0.0;
                if (forcing) {
                    const double *fc = forcing + (size_t)c * D::NRHS;
                    for (int col = 0; col < D::NRHS; ++col) v += Km[(size_t)i * LD + N + col] * fc[col];
                }
                for (int x = 0; x < NUH; ++x)
                    if (x < 4 * NF || x >= NRT) v -= Km[(size_t)i * LD + x] * Xs[x];
                Km[(size_t)i * LD + N] = v;
            }
            __syncthreads();
        }
        // eliminate the interior RT unknowns, then the mean-free pressure
        for (int t = 0; t < (NRT - 4 * NF) + (NPK - 1); ++t) {
            const int q = t < NRT - 4 * NF ? 4 * NF + t : NUH + 1 + (t - (NRT - 4 * NF));
            const double piv = Km[(size_t)q * LD + q];
            if (tid == 0 && (!(fabs(piv) > 1e-300) || !isfinite(piv))) bad = 1;
            const double pinv = 1.0 / piv;
            for (int i = tid; i < N; i += nt) colq[i] = Km[(size_t)i * LD + q];
            for (int j = tid; j < LD; j += nt) rowq[j] = Km[(size_t)q * LD + j] * pinv;
            __syncthreads();
            for (int idx = tid; idx < N * LD; idx += nt) {
                const int i = idx / LD, j = idx % LD;
                if (i == q) continue;
                Km[idx] = fma(-colq[i], rowq[j], Km[idx]);
            }
            __syncthreads();
        }
        if (bad) {
            if (tid == 0) atomicOr(flag, 1);
            __syncthreads();
            continue;
        }
        if (rec.x) {
            // interior RT coefficients from the eliminated local rows, then the outputs
            for (int t = tid; t < NRT - 4 * NF; t += nt) {
                const int q = 4 * NF + t;
                Xs[q] = Km[(size_t)q * LD + N] / Km[(size_t)q * LD + q];
            }
            __syncthreads();
            if (rec.rt)
                for (int i = tid; i < NRT; i += nt) rec.rt[(size_t)c * NRT + i] = Xs[i];
            if (rec.L)   // L = -(nu/|det J|) B x: coefficients of component (c, e) over g_j
                for (int r = tid; r < 9 * NPK; r += nt) {
                    double v = 0.0;
                    for (int x = 0; x < NUH; ++x) v += Bm[(size_t)r * NUH + x] * Xs[x];
                    rec.L[(size_t)c * 9 * NPK + r] = -(nuc / adet) * v;
                }
            if (rec.ulat)   // u_h = J u^ / |det J| at the lattice
                for (int idx = tid; idx < NLAT * 3; idx += nt) {
                    const int n = idx / 3, a = idx % 3;
                    double w[3] = {0.0, 0.0, 0.0};
                    for (int i = 0; i < NRT; ++i)
                        for (int b = 0; b < 3; ++b) w[b] += Xs[i] * R7[((size_t)n * NRT + i) * 3 + b];
                    rec.ulat[(size_t)c * NLAT * 3 + idx] = (J[a][0] * w[0] + J[a][1] * w[1] + J[a][2] * w[2]) / adet;
                }
            __syncthreads();
            continue;
        }
        // gather the global block in the per-face layout [normal | t1 | t2], rotate the normal
        // rows and columns, add the AL term
        auto gidx = [&](int g) {
            const int f = g / DPF, t = g % DPF;
            return t < NF ? f * NF + t : NRT + f * 2 * NF + (t - NF);
        };
        auto tf = [&](int f, int m, int m2) {
            return fsig[f] * sqrt(farea[f]) * Q[((size_t)fperm[f] * NF + m) * NF + m2];
        };
        for (int idx = tid; idx < NLOC * (NLOC + D::NRHS); idx += nt) {
            const int g1 = idx / (NLOC + D::NRHS), col = idx % (NLOC + D::NRHS);
            const int kc = col < NLOC ? gidx(col) : N + (col - NLOC);
            const int f = g1 / DPF, t = g1 % DPF;
            double v;
            if (t < NF) {
                v = 0.0;
                for (int m2 = 0; m2 < NF; ++m2) v += tf(f, t, m2) * Km[(size_t)gidx(f * DPF + m2) * LD + kc];
            } else {
                v = Km[(size_t)gidx(g1) * LD + kc];
            }
            Rm[idx] = v;
        }
        __syncthreads();
        const double al = gamma * nuc / (adet / 6.0);
        for (int idx = tid; Aout && idx < NLOC * NLOC; idx += nt) {
            const int g1 = idx / NLOC, g2 = idx % NLOC;
            const int f = g2 / DPF, t = g2 % DPF;
            const double *row = Rm + (size_t)g1 * (NLOC + D::NRHS);
            double v;
            if (t < NF) {
                v = 0.0;
                for (int m2 = 0; m2 < NF; ++m2) v += tf(f, t, m2) * row[f * DPF + m2];
            } else {
                v = row[g2];
            }
            const int f1 = g1 / DPF, t1i = g1 % DPF;
            if (t1i == 0 && t == 0) v += al * fsig[f1] * sqrt(farea[f1]) * fsig[f] * sqrt(farea[f]);
            const int lf = g1 / DPF, d = g1 % DPF;
            const size_t o = (size_t)c * NLOC * NLOC + (size_t)lf * NLOC * DPF + (size_t)g2 * DPF + d;
            Aout[o] = v;
            if (Af) Af[o] = (float)v;
        }
        if (Fel) {
            for (int g1 = tid; g1 < NLOC; g1 += nt) {
                const double *row = Rm + (size_t)g1 * (NLOC + D::NRHS) + NLOC;
                double v = 0.0;
                if (forcing) {
                    const double *fc = forcing + (size_t)c * D::NRHS;
                    for (int col = 0; col < D::NRHS; ++col) v += row[col] * fc[col];
                }
                Fel[(size_t)c * NLOC + g1] = v;
            }
        }
        __syncthreads();
    }
}

// Harmonic extension of eq. harmonic-ex per coarse cell: the rows of the eight children's
// lowest-order matrices that belong to the faces inside the cell (T) against all local faces
// (16 B slots, then the 8 T slots, 3 unknowns each), Gauss-Jordan on the SPD block A_TT, and
// H = -A_TT^-1 A_TB [24][48]
__global__ void __launch_bounds__(64)
transfer_H3_kernel(int64_t ncc, const int *__restrict__ children, const int *__restrict__ child_slot,
                   const double *__restrict__ A0, double *__restrict__ H, float *__restrict__ Hf, int *flag) {
    constexpr int NT = 3 * TR3_T, NC = 3 * TR3_SLOTS;
    __shared__ double M[NT][NC];
    __shared__ double rowp[NC], colp[NT];
    __shared__ int ok;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int64_t P = blockIdx.x; P < ncc; P += gridDim.x) {
        for (int i = tid; i < NT * NC; i += nt) (&M[0][0])[i] = 0.0;
        if (tid == 0) ok = 1;
        __syncthreads();
        if (tid == 0)
            for (int ch = 0; ch < 8; ++ch) {
                const int c = children[8 * P + ch];
                const int *cs = child_slot + 32 * P + 4 * ch;
                for (int lf = 0; lf < 4; ++lf) {
                    const int s1 = cs[lf];
                    if (s1 < TR3_B) continue;   // B rows are not needed; -1: boundary
                    for (int d = 0; d < 3; ++d)
                        for (int lf2 = 0; lf2 < 4; ++lf2) {
                            const int s2 = cs[lf2];
                            if (s2 < 0) continue;
                            for (int d2 = 0; d2 < 3; ++d2)
                                M[3 * (s1 - TR3_B) + d][3 * s2 + d2] += A0[(size_t)c * 144 + lf * 36 + (lf2 * 3 + d2) * 3 + d];
                        }
                }
            }
        __syncthreads();
        for (int piv = 0; piv < NT; ++piv) {
            const double pv = M[piv][3 * TR3_B + piv];
            if (tid == 0 && !(pv > 0.0)) ok = 0;
            const double pinv = pv > 0.0 ? 1.0 / pv : 0.0;
            for (int j = tid; j < NC; j += nt) rowp[j] = M[piv][j] * pinv;
            for (int i = tid; i < NT; i += nt) colp[i] = M[i][3 * TR3_B + piv];
            __syncthreads();
            for (int idx = tid; idx < NT * NC; idx += nt) {
                const int i = idx / NC, j = idx % NC;
                M[i][j] = i == piv ? rowp[j] : fma(-colp[i], rowp[j], M[i][j]);
            }
            __syncthreads();
        }
        for (int idx = tid; idx < NT * 3 * TR3_B; idx += nt) {
            const int t = idx / (3 * TR3_B), c = idx % (3 * TR3_B);
            const double v = -M[t][c];
            H[(size_t)P * NT * 3 * TR3_B + idx] = v;
            if (Hf) Hf[(size_t)P * NT * 3 * TR3_B + idx] = (float)v;
        }
        if (tid == 0 && !ok) atomicOr(flag, 4);
        __syncthreads();
    }
}

// Patch inverses of the edge patches (Section 3.4.2): A_ss assembled from the star cells'
// element matrices (two cells per patch face), inverted by Gauss-Jordan with the SPD pivots
// checked positive, stored transposed (Pinv[p][j][i] = (A_ss^-1)_ij) for the sweep.  The patch
// matrix lives in a global workspace slice per block (an order-3 edge patch has 180 unknowns,
// 259 KB in FP64, more than a block's shared memory).
__global__ void __launch_bounds__(256)
patch_inverse3_kernel(int n_patches, int pf_max, int pc_max, int dpf, int nloc, int np_max,
                      const int *__restrict__ patch_nf, const int *__restrict__ patch_nc,
                      const int *__restrict__ patch_cells, const int *__restrict__ slot_src,
                      const double *__restrict__ A, double *__restrict__ Pinv, float *__restrict__ Pinvf,
                      double *__restrict__ scratch, int *flag) {
    extern __shared__ double sm3[];
    double *colp = sm3;                          // np_max
    double *rowp = colp + np_max;                // np_max
    int *lfmap = (int *)(rowp + np_max);         // pc_max * pf_max
    double *M = scratch + (size_t)blockIdx.x * np_max * np_max;
    __shared__ int ok;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int p = blockIdx.x; p < n_patches; p += gridDim.x) {
        const int nf = patch_nf[p], ncell = patch_nc[p], np = nf * dpf;
        for (int i = tid; i < pc_max * pf_max; i += nt) lfmap[i] = -1;
        if (tid == 0) ok = 1;
        __syncthreads();
        if (tid == 0)
            for (int j = 0; j < nf; ++j)
                for (int q = 0; q < 2; ++q) {
                    const int src = slot_src[((size_t)p * pf_max + j) * 2 + q];
                    lfmap[(src >> 2) * pf_max + j] = src & 3;
                }
        __syncthreads();
        for (int idx = tid; idx < np * np; idx += nt) {
            const int P = idx / np, Q = idx % np;
            const int j1 = P / dpf, d1 = P % dpf, j2 = Q / dpf, d2 = Q % dpf;
            double v = 0.0;
            for (int si = 0; si < ncell; ++si) {
                const int l1 = lfmap[si * pf_max + j1], l2 = lfmap[si * pf_max + j2];
                if (l1 < 0 || l2 < 0) continue;
                const int c = patch_cells[(size_t)p * pc_max + si];
                v += A[(size_t)c * nloc * nloc + (size_t)l1 * nloc * dpf + (size_t)(l2 * dpf + d2) * dpf + d1];
            }
            M[idx] = v;
        }
        __syncthreads();
        for (int piv = 0; piv < np; ++piv) {
            const double d = M[(size_t)piv * np + piv];
            if (tid == 0 && !(d > 0.0)) ok = 0;
            const double dinv = d > 0.0 ? 1.0 / d : 1.0;
            for (int i = tid; i < np; i += nt) {
                colp[i] = M[(size_t)i * np + piv];
                rowp[i] = M[(size_t)piv * np + i] * dinv;
            }
            __syncthreads();
            for (int i = tid >> 5; i < np; i += nt >> 5) {
                const double ci = colp[i];
                for (int j = tid & 31; j < np; j += 32) {
                    double v;
                    if (i == piv) v = (j == piv) ? dinv : rowp[j];
                    else if (j == piv) v = -ci * dinv;
                    else v = fma(-ci, rowp[j], M[(size_t)i * np + j]);
                    M[(size_t)i * np + j] = v;
                }
            }
            __syncthreads();
        }
        for (int idx = tid; idx < np_max * np_max; idx += nt) {
            const int j = idx / np_max, i = idx % np_max;
            const double v = (i < np && j < np) ? M[(size_t)i * np + j] : 0.0;
            if (Pinv) Pinv[(size_t)p * np_max * np_max + idx] = v;
            if (Pinvf) Pinvf[(size_t)p * np_max * np_max + idx] = (float)v;
        }
        if (tid == 0 && !ok) atomicOr(flag, 2);
        __syncthreads();
    }
}

} // namespace

size_t condense3_scratch_doubles(int k, int blocks) {
    switch (k) {
    case 0: return (size_t)blocks * Dims3<0>::SCR;
    case 1: return (size_t)blocks * Dims3<1>::SCR;
    case 2: return (size_t)blocks * Dims3<2>::SCR;
    case 3: return (size_t)blocks * Dims3<3>::SCR;
    default: return 0;
    }
}

cudaError_t launch_condense3(int k, const DevLevel &L, const double *ref, const RefTables3 &rt, double nu,
                             const double *nu_cell, double beta, double gamma, const double *forcing, double *A,
                             float *Af, double *Fel, double *scratch, int blocks, int *flag, cudaStream_t s,
                             const Recover3 &rec) {
    (void)rt;
    if (L.nc == 0) return cudaSuccess;
    const unsigned nb = (unsigned)std::min<int64_t>(L.nc, blocks);
    note_launches(1);
#define HDG_C3(KK)                                                                                               \
    case KK:                                                                                                     \
        condense3_kernel<KK><<<nb, 128, 0, s>>>(L.nc, L.coords.p, L.cells.p, ref, nu, nu_cell, beta, gamma,       \
                                                forcing, A, Af, Fel, L.cell_d.p, L.cell_area.p, scratch, flag,  \
                                                rec);                                                     \
        break;
    switch (k) {
        HDG_C3(0)
        HDG_C3(1)
        HDG_C3(2)
        HDG_C3(3)
    default: return cudaErrorInvalidValue;
    }
#undef HDG_C3
    return cudaGetLastError();
}

cudaError_t launch_transfer_H3(const DevLevel &F, int *flag, cudaStream_t s) {
    if (F.nc_coarse == 0) return cudaSuccess;
    note_launches(1);
    transfer_H3_kernel<<<(unsigned)std::min<int64_t>(F.nc_coarse, 4096), 64, 0, s>>>(
        F.nc_coarse, F.tr_children.p, F.tr_child_slot.p, F.op0.A.p, F.tr_H.p, F.tr_Hf.p, flag);
    return cudaGetLastError();
}

size_t patch_inverse3_scratch_doubles(const DevLevel &L, const DevOperator &op, int blocks) {
    return (size_t)std::min<int64_t>(std::max(L.n_patches, 1), blocks) * op.np_max * op.np_max;
}

cudaError_t launch_patch_inverse3(const DevLevel &L, const DevOperator &op, double *scratch, int blocks, int *flag,
                                  cudaStream_t s) {
    if (L.n_patches == 0) return cudaSuccess;
    const unsigned nb = (unsigned)std::min(L.n_patches, blocks);
    const size_t smem = sizeof(double) * 2 * op.np_max + sizeof(int) * (size_t)L.pc_max * L.pf_max;
    note_launches(1);
    patch_inverse3_kernel<<<nb, 256, smem, s>>>(L.n_patches, L.pf_max, L.pc_max, op.dpf, op.nloc, op.np_max,
                                                L.patch_nf.p, L.patch_nc.p, L.patch_cells.p, L.patch_slot_src.p,
                                                op.A.p, op.Pinv.p, op.Pinvf.p, scratch, flag);
    return cudaGetLastError();
}

} // namespace hdg
