// Reference-tetrahedron tables for the device-side static condensation in 3D.
//
// On an affine tetrahedron x = X0 + J x^ every integral of the local H(div)-HDG system
// (eq. stWeak, d = 3) is a contraction of integrals on the reference tetrahedron
// K^ = {x, y, z >= 0, x + y + z <= 1} with J (contravariant Piola map u = J u^ / |det J|
// for the Raviart-Thomas space, which keeps outward fluxes; composition for the
// polynomial spaces).  The integrals are exact: functions are polynomials held as
// monomial coefficients and integrated by the Dirichlet formulas
//   ∫_K^ x^a y^b z^c = a! b! c! / (a+b+c+3)!,   ∫_T λ0^a λ1^b λ2^c dA = 2|T| a! b! c! / (a+b+c+2)!.
//
// Bases on K^ (barycentrics λ0 = 1-x-y-z, λ1 = x, λ2 = y, λ3 = z; face f opposite vertex f
// with canonical vertices in ascending local order a < b < c, outward unit normal n^_f):
//   g_j    orthonormal basis of P^k(K^) (Gram-Schmidt on monomials by degree), g_0 constant;
//   l_m    canonical face basis of face f: Gram-Schmidt of λ_b^i λ_c^j (i + j <= k, by degree
//          then j), orthonormal for the measure dS/|F^_f|;
//   phi_i  RT_k(K^) = [P^k]^3 + x P~^k, dual to N_{f,m}(v) = ∫_F^f (v.n^_f) l_m dS (i = f nf + m)
//          and I_{a,r}(v) = ∫ v_a g_r (a = 1..3, r < dim P^{k-1});
//   lam_n  Lagrange basis of P^{k+1} on the lattice of the forcing layout.
// Tables:
//   R1[i][a][b][j] = ∫ d_b phi_{i,a} g_j          R4[i][a][i'][b] = ∫ phi_{i,a} phi_{i',b}
//   R2[f][i][a][j] = ∫_F^f phi_{i,a} g_j dS       R5[i][j]        = ∫ div phi_i g_j
//   R3[f][j][m]    = ∫_F^f g_j l_m dS             R6[i][a][n]     = ∫ phi_{i,a} lam_n
//   Q[p][m][m']    = (1/|F^|) ∫_F^ l^p_m l_m' dS: the face basis built on the vertex order p
//                    (one of the 6 orders of the canonical vertices, index of (s0, s1, s2) in
//                    lexicographic order) against the canonical one; orthogonal, the same
//                    for every face
//   FA[f]          = |F^_f|
//   R7[n][i][a]    = phi_{i,a} at lattice point n
// Post-processing (eq. stPost, not packed with the above):
//   P1[(a*3+b)][n][n'] = ∫ d_a lam_n d_b lam_n'   P2[j][n][b] = ∫ g_j d_b lam_n   P3[n] = ∫ lam_n
#include <algorithm>
#include <cmath>
#include <stdexcept>
#include <vector>

#include "hdg3d_internal.h"

namespace hdg {
namespace {

// polynomial in (x, y, z) of total degree <= deg; coefficient of x^a y^b z^c at a dense
// (deg+1)^3 index (entries with a + b + c > deg stay zero)
struct P3 {
    int deg = 0;
    std::vector<double> c;
    explicit P3(int d = 0) : deg(d), c((size_t)(d + 1) * (d + 1) * (d + 1), 0.0) {}
    int idx(int a, int b, int e) const { return (a * (deg + 1) + b) * (deg + 1) + e; }
    double &at(int a, int b, int e) { return c[idx(a, b, e)]; }
    double get(int a, int b, int e) const {
        return (a >= 0 && b >= 0 && e >= 0 && a + b + e <= deg) ? c[idx(a, b, e)] : 0.0;
    }
};

P3 mul(const P3 &p, const P3 &q) {
    P3 r(p.deg + q.deg);
    for (int a = 0; a <= p.deg; ++a)
        for (int b = 0; a + b <= p.deg; ++b)
            for (int e = 0; a + b + e <= p.deg; ++e) {
                const double pv = p.c[p.idx(a, b, e)];
                if (pv == 0.0) continue;
                for (int a2 = 0; a2 <= q.deg; ++a2)
                    for (int b2 = 0; a2 + b2 <= q.deg; ++b2)
                        for (int e2 = 0; a2 + b2 + e2 <= q.deg; ++e2) {
                            const double qv = q.c[q.idx(a2, b2, e2)];
                            if (qv != 0.0) r.at(a + a2, b + b2, e + e2) += pv * qv;
                        }
            }
    return r;
}

P3 axpy(const P3 &p, const P3 &q, double s) {   // p + s q
    P3 r(std::max(p.deg, q.deg));
    for (int a = 0; a <= r.deg; ++a)
        for (int b = 0; a + b <= r.deg; ++b)
            for (int e = 0; a + b + e <= r.deg; ++e) r.at(a, b, e) = p.get(a, b, e) + s * q.get(a, b, e);
    return r;
}

P3 deriv(const P3 &p, int dir) {
    P3 r(std::max(p.deg - 1, 0));
    for (int a = 0; a <= p.deg; ++a)
        for (int b = 0; a + b <= p.deg; ++b)
            for (int e = 0; a + b + e <= p.deg; ++e) {
                const double v = p.c[p.idx(a, b, e)];
                if (v == 0.0) continue;
                if (dir == 0 && a > 0) r.at(a - 1, b, e) += a * v;
                if (dir == 1 && b > 0) r.at(a, b - 1, e) += b * v;
                if (dir == 2 && e > 0) r.at(a, b, e - 1) += e * v;
            }
    return r;
}

P3 mono(int a, int b, int e) {
    P3 p(a + b + e);
    p.at(a, b, e) = 1.0;
    return p;
}

double fact(int n) {
    double r = 1.0;
    for (int i = 2; i <= n; ++i) r *= i;
    return r;
}

double integrate_tet(const P3 &p) {
    double s = 0.0;
    for (int a = 0; a <= p.deg; ++a)
        for (int b = 0; a + b <= p.deg; ++b)
            for (int e = 0; a + b + e <= p.deg; ++e) {
                const double v = p.c[p.idx(a, b, e)];
                if (v != 0.0) s += v * fact(a) * fact(b) * fact(e) / fact(a + b + e + 3);
            }
    return s;
}

// ∫ over reference face f (opposite vertex f) with respect to its area element
double integrate_face(const P3 &p, int f) {
    double s = 0.0;
    for (int a = 0; a <= p.deg; ++a)
        for (int b = 0; a + b <= p.deg; ++b)
            for (int e = 0; a + b + e <= p.deg; ++e) {
                const double v = p.c[p.idx(a, b, e)];
                if (v == 0.0) continue;
                if (f == 0) {
                    // x + y + z = 1: x, y, z are the face's barycentrics, dS = sqrt(3) dy dz
                    s += v * std::sqrt(3.0) * fact(a) * fact(b) * fact(e) / fact(a + b + e + 2);
                } else if (f == 1) {
                    if (a == 0) s += v * fact(b) * fact(e) / fact(b + e + 2);
                } else if (f == 2) {
                    if (b == 0) s += v * fact(a) * fact(e) / fact(a + e + 2);
                } else {
                    if (e == 0) s += v * fact(a) * fact(b) / fact(a + b + 2);
                }
            }
    return s;
}

double eval(const P3 &p, double x, double y, double z) {
    double s = 0.0;
    for (int a = 0; a <= p.deg; ++a)
        for (int b = 0; a + b <= p.deg; ++b)
            for (int e = 0; a + b + e <= p.deg; ++e) {
                const double v = p.c[p.idx(a, b, e)];
                if (v != 0.0) s += v * std::pow(x, a) * std::pow(y, b) * std::pow(z, e);
            }
    return s;
}

P3 barycentric(int v) {
    P3 p(1);
    if (v == 0) {
        p.at(0, 0, 0) = 1.0;
        p.at(1, 0, 0) = p.at(0, 1, 0) = p.at(0, 0, 1) = -1.0;
    } else {
        p.at(v == 1, v == 2, v == 3) = 1.0;
    }
    return p;
}

P3 power(const P3 &p, int n) {
    P3 r = mono(0, 0, 0);
    for (int i = 0; i < n; ++i) r = mul(r, p);
    return r;
}

// exponents (a, b, c) of P^deg by total degree (the same order as the host's 3D ordering)
std::vector<std::array<int, 3>> exps(int deg) {
    std::vector<std::array<int, 3>> out;
    for (int n = 0; n <= deg; ++n)
        for (int e = 0; e <= n; ++e)
            for (int b = 0; b <= n - e; ++b) out.push_back({n - b - e, b, e});
    return out;
}

// dense inverse (Gauss-Jordan with partial pivoting)
std::vector<double> invert(std::vector<double> A, int n) {
    std::vector<double> I((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) I[(size_t)i * n + i] = 1.0;
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(A[(size_t)r * n + c]) > std::fabs(A[(size_t)p * n + c])) p = r;
        if (std::fabs(A[(size_t)p * n + c]) < 1e-300) throw std::runtime_error("singular 3D reference matrix");
        for (int j = 0; j < n; ++j) {
            std::swap(A[(size_t)c * n + j], A[(size_t)p * n + j]);
            std::swap(I[(size_t)c * n + j], I[(size_t)p * n + j]);
        }
        const double d = A[(size_t)c * n + c];
        for (int j = 0; j < n; ++j) {
            A[(size_t)c * n + j] /= d;
            I[(size_t)c * n + j] /= d;
        }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            const double f = A[(size_t)r * n + c];
            if (f == 0.0) continue;
            for (int j = 0; j < n; ++j) {
                A[(size_t)r * n + j] -= f * A[(size_t)c * n + j];
                I[(size_t)r * n + j] -= f * I[(size_t)c * n + j];
            }
        }
    }
    return I;
}

// lower Cholesky factor of an SPD matrix, then its inverse (row m = coefficients of the
// m-th Gram-Schmidt function over the input functions)
std::vector<double> gram_schmidt_coeffs(const std::vector<double> &G, int n) {
    std::vector<double> L((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = G[(size_t)i * n + j];
            for (int q = 0; q < j; ++q) s -= L[(size_t)i * n + q] * L[(size_t)j * n + q];
            if (i == j) {
                if (!(s > 0)) throw std::runtime_error("3D reference Gram matrix not positive definite");
                L[(size_t)i * n + i] = std::sqrt(s);
            } else {
                L[(size_t)i * n + j] = s / L[(size_t)j * n + j];
            }
        }
    return invert(L, n);
}

const int FV3[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
const int PERM3[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

// orthonormal face basis (measure dS/|F^_f|) from λ_v1^i λ_v2^j, v1, v2 local vertices
std::vector<P3> face_basis(int k, int f, int v1, int v2, double area) {
    std::vector<P3> mon;
    const P3 l1 = barycentric(v1), l2 = barycentric(v2);
    for (int n = 0; n <= k; ++n)
        for (int j = 0; j <= n; ++j) mon.push_back(mul(power(l1, n - j), power(l2, j)));
    const int nf = (int)mon.size();
    std::vector<double> G((size_t)nf * nf);
    for (int r = 0; r < nf; ++r)
        for (int s = 0; s < nf; ++s) G[(size_t)r * nf + s] = integrate_face(mul(mon[r], mon[s]), f) / area;
    std::vector<double> C = gram_schmidt_coeffs(G, nf);
    std::vector<P3> out;
    for (int m = 0; m < nf; ++m) {
        P3 p(k);
        for (int r = 0; r <= m; ++r) p = axpy(p, mon[r], C[(size_t)m * nf + r]);
        out.push_back(p);
    }
    return out;
}

} // namespace

void build_reference_tables_3d(int k, RefTables3 &T) {
    if (k < 0 || k > MAX_K3) throw std::runtime_error("3D reference tables: k out of range");
    T = RefTables3();
    T.k = k;
    const double FA[4] = {std::sqrt(3.0) / 2.0, 0.5, 0.5, 0.5};
    const double NRM[4][3] = {{1 / std::sqrt(3.0), 1 / std::sqrt(3.0), 1 / std::sqrt(3.0)},
                              {-1, 0, 0}, {0, -1, 0}, {0, 0, -1}};
    // g_j: orthonormal P^k on K^
    const auto E = exps(k);
    const int npk = (int)E.size();
    std::vector<P3> gm;
    for (auto &e : E) gm.push_back(mono(e[0], e[1], e[2]));
    std::vector<double> G((size_t)npk * npk);
    for (int r = 0; r < npk; ++r)
        for (int s = 0; s < npk; ++s) G[(size_t)r * npk + s] = integrate_tet(mul(gm[r], gm[s]));
    std::vector<double> Cg = gram_schmidt_coeffs(G, npk);
    std::vector<P3> g;
    for (int j = 0; j < npk; ++j) {
        P3 p(k);
        for (int r = 0; r <= j; ++r) p = axpy(p, gm[r], Cg[(size_t)j * npk + r]);
        g.push_back(p);
    }
    const int npk1 = k >= 1 ? (int)exps(k - 1).size() : 0;
    // canonical face bases
    const int nf = (k + 1) * (k + 2) / 2;
    std::vector<std::vector<P3>> lf(4);
    for (int f = 0; f < 4; ++f) lf[f] = face_basis(k, f, FV3[f][1], FV3[f][2], FA[f]);
    // RT_k spanning set (a basis): m e_a for m in P^k, x m~ for m~ homogeneous of degree k
    std::vector<std::array<P3, 3>> span;
    for (auto &e : E)
        for (int a = 0; a < 3; ++a) {
            std::array<P3, 3> v = {P3(k + 1), P3(k + 1), P3(k + 1)};
            v[a].at(e[0], e[1], e[2]) = 1.0;
            span.push_back(v);
        }
    for (auto &e : E) {
        if (e[0] + e[1] + e[2] != k) continue;
        std::array<P3, 3> v = {P3(k + 1), P3(k + 1), P3(k + 1)};
        v[0].at(e[0] + 1, e[1], e[2]) = 1.0;
        v[1].at(e[0], e[1] + 1, e[2]) = 1.0;
        v[2].at(e[0], e[1], e[2] + 1) = 1.0;
        span.push_back(v);
    }
    const int nrt = (int)span.size();
    if (nrt != (k + 1) * (k + 2) * (k + 4) / 2 || 4 * nf + 3 * npk1 != nrt)
        throw std::runtime_error("3D RT dimension mismatch");
    std::vector<double> V((size_t)nrt * nrt);
    for (int s = 0; s < nrt; ++s) {
        int row = 0;
        for (int f = 0; f < 4; ++f) {
            P3 vn(k + 1);
            for (int a = 0; a < 3; ++a) vn = axpy(vn, span[s][a], NRM[f][a]);
            for (int m = 0; m < nf; ++m) V[(size_t)(row++) * nrt + s] = integrate_face(mul(vn, lf[f][m]), f);
        }
        for (int a = 0; a < 3; ++a)
            for (int r = 0; r < npk1; ++r) V[(size_t)(row++) * nrt + s] = integrate_tet(mul(span[s][a], g[r]));
    }
    std::vector<double> Vi = invert(V, nrt);
    std::vector<std::array<P3, 3>> phi(nrt);
    for (int i = 0; i < nrt; ++i) {
        std::array<P3, 3> v = {P3(k + 1), P3(k + 1), P3(k + 1)};
        for (int s = 0; s < nrt; ++s) {
            const double w = Vi[(size_t)s * nrt + i];
            if (w == 0.0) continue;
            for (int a = 0; a < 3; ++a) v[a] = axpy(v[a], span[s][a], w);
        }
        phi[i] = v;
    }
    // Lagrange basis of P^{k+1} on the forcing lattice
    const int q = k + 1;
    std::vector<std::array<double, 3>> pts;
    for (int a3 = 0; a3 <= q; ++a3)
        for (int a2 = 0; a2 <= q - a3; ++a2)
            for (int a1 = 0; a1 <= q - a2 - a3; ++a1) pts.push_back({a1 / double(q), a2 / double(q), a3 / double(q)});
    const auto El = exps(q);
    const int nlat = (int)pts.size();
    std::vector<double> Vd((size_t)nlat * nlat);
    for (int n = 0; n < nlat; ++n)
        for (int r = 0; r < nlat; ++r)
            Vd[(size_t)n * nlat + r] = std::pow(pts[n][0], El[r][0]) * std::pow(pts[n][1], El[r][1]) *
                                       std::pow(pts[n][2], El[r][2]);
    std::vector<double> Vdi = invert(Vd, nlat);
    std::vector<P3> lam;
    for (int n = 0; n < nlat; ++n) {
        P3 p(q);
        for (int r = 0; r < nlat; ++r) p.at(El[r][0], El[r][1], El[r][2]) = Vdi[(size_t)r * nlat + n];
        lam.push_back(p);
    }
    T.npk = npk;
    T.nrt = nrt;
    T.nf = nf;
    T.nlat = nlat;
    // tables
    T.R1.assign((size_t)nrt * 9 * npk, 0.0);
    for (int i = 0; i < nrt; ++i)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                const P3 d = deriv(phi[i][a], b);
                for (int j = 0; j < npk; ++j)
                    T.R1[(((size_t)i * 3 + a) * 3 + b) * npk + j] = integrate_tet(mul(d, g[j]));
            }
    T.R2.assign((size_t)4 * nrt * 3 * npk, 0.0);
    for (int f = 0; f < 4; ++f)
        for (int i = 0; i < nrt; ++i)
            for (int a = 0; a < 3; ++a)
                for (int j = 0; j < npk; ++j)
                    T.R2[(((size_t)f * nrt + i) * 3 + a) * npk + j] = integrate_face(mul(phi[i][a], g[j]), f);
    T.R3.assign((size_t)4 * npk * nf, 0.0);
    for (int f = 0; f < 4; ++f)
        for (int j = 0; j < npk; ++j)
            for (int m = 0; m < nf; ++m)
                T.R3[((size_t)f * npk + j) * nf + m] = integrate_face(mul(g[j], lf[f][m]), f);
    T.R4.assign((size_t)nrt * 3 * nrt * 3, 0.0);
    for (int i = 0; i < nrt; ++i)
        for (int a = 0; a < 3; ++a)
            for (int i2 = i; i2 < nrt; ++i2)
                for (int b = 0; b < 3; ++b) {
                    const double v = integrate_tet(mul(phi[i][a], phi[i2][b]));
                    T.R4[(((size_t)i * 3 + a) * nrt + i2) * 3 + b] = v;
                    T.R4[(((size_t)i2 * 3 + b) * nrt + i) * 3 + a] = v;
                }
    T.R5.assign((size_t)nrt * npk, 0.0);
    for (int i = 0; i < nrt; ++i) {
        const P3 dv = axpy(axpy(deriv(phi[i][0], 0), deriv(phi[i][1], 1), 1.0), deriv(phi[i][2], 2), 1.0);
        for (int j = 0; j < npk; ++j) T.R5[(size_t)i * npk + j] = integrate_tet(mul(dv, g[j]));
    }
    T.R6.assign((size_t)nrt * 3 * nlat, 0.0);
    for (int i = 0; i < nrt; ++i)
        for (int a = 0; a < 3; ++a)
            for (int n = 0; n < nlat; ++n) T.R6[((size_t)i * 3 + a) * nlat + n] = integrate_tet(mul(phi[i][a], lam[n]));
    // face-order transforms, computed on face 3 (canonical vertices 0, 1, 2)
    T.Q.assign((size_t)6 * nf * nf, 0.0);
    for (int p = 0; p < 6; ++p) {
        const std::vector<P3> lp = face_basis(k, 3, FV3[3][PERM3[p][1]], FV3[3][PERM3[p][2]], FA[3]);
        for (int m = 0; m < nf; ++m)
            for (int m2 = 0; m2 < nf; ++m2)
                T.Q[((size_t)p * nf + m) * nf + m2] = integrate_face(mul(lp[m], lf[3][m2]), 3) / FA[3];
    }
    T.FA.assign(FA, FA + 4);
    // post-processing tables of eq. stPost
    std::vector<std::array<P3, 3>> dlam(nlat);
    for (int n = 0; n < nlat; ++n)
        for (int a = 0; a < 3; ++a) dlam[n][a] = deriv(lam[n], a);
    T.P1.assign((size_t)9 * nlat * nlat, 0.0);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            for (int n1 = 0; n1 < nlat; ++n1)
                for (int n2 = 0; n2 < nlat; ++n2)
                    T.P1[((size_t)(a * 3 + b) * nlat + n1) * nlat + n2] = integrate_tet(mul(dlam[n1][a], dlam[n2][b]));
    T.P2.assign((size_t)npk * nlat * 3, 0.0);
    for (int j = 0; j < npk; ++j)
        for (int n = 0; n < nlat; ++n)
            for (int b = 0; b < 3; ++b) T.P2[((size_t)j * nlat + n) * 3 + b] = integrate_tet(mul(g[j], dlam[n][b]));
    T.P3.assign((size_t)nlat, 0.0);
    for (int n = 0; n < nlat; ++n) T.P3[n] = integrate_tet(lam[n]);
    // R7[n][i][a] = phi_{i,a} at lattice point n (recovery of u_h at the forcing lattice)
    T.R7.assign((size_t)nlat * nrt * 3, 0.0);
    for (int n = 0; n < nlat; ++n)
        for (int i = 0; i < nrt; ++i)
            for (int a = 0; a < 3; ++a)
                T.R7[((size_t)n * nrt + i) * 3 + a] = eval(phi[i][a], pts[n][0], pts[n][1], pts[n][2]);
}

std::vector<double> pack_reference_tables_3d(const RefTables3 &T) {
    std::vector<double> out;
    for (const std::vector<double> *t : {&T.R1, &T.R2, &T.R3, &T.R4, &T.R5, &T.R6, &T.Q, &T.FA, &T.R7})
        out.insert(out.end(), t->begin(), t->end());
    return out;
}

} // namespace hdg
