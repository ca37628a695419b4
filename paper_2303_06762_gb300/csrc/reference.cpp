// Reference-element tables for the device-side static condensation.
//
// All cell integrals of the local H(div)-HDG system (eq. stWeak) on an affine
// triangle are contractions of integrals on the reference triangle
// K^ = {x, y >= 0, x + y <= 1} with the element Jacobian (Piola map for the
// Raviart-Thomas space, composition for the polynomial spaces).  This file
// builds those reference integrals with a collapsed (Duffy) Gauss-Legendre
// rule of k+5 nodes per direction (exact for every integrand here, degree
// <= 2k+2), functions being held as coefficients over monomials centred at
// the centroid, (x-1/3)^a (y-1/3)^b, which keeps the coefficients of the
// degree-(k+1) dual bases small.
//
// Spaces (Section 2) and bases on K^:
//   g_j   orthonormal basis of P^k(K^) (Gram–Schmidt on monomials by degree),
//         g_0 = sqrt(2) constant, g_j (j >= 1) of zero mean;
//   phi_i basis of RT_k(K^) = [P^k]^2 + x P~^k dual to the degrees of freedom
//         N_{f,m}(v) = ∫_{F^_f} (v.n^_f) l_m(s) ds^   (m = 0..k, s from the lower
//         to the higher local vertex of facet f, l_m(s) = sqrt(2m+1) P_m(2s-1)),
//         I_{a,r}(v) = ∫_K^ v_a g_r   (a = 1,2, r < dim P^{k-1});
//   lam_n Lagrange basis of P^{k+1} on the lattice of the forcing layout.
// Tables:
//   R1[i][a][b][j] = ∫ d_b phi_{i,a} g_j          R4[i][a][i'][b] = ∫ phi_{i,a} phi_{i',b}
//   R2[f][i][a][j] = ∫_{F^_f} phi_{i,a} g_j ds^   R5[i][j] = ∫ div phi_i g_j
//   R3[f][j][m]    = ∫_0^1 g_j(x_f(s)) l_m(s) ds  R6[i][a][n] = ∫ phi_{i,a} lam_n
//   R7[i][a][n]    = phi_{i,a} at lattice point n  R8[n][n'] = ∫ lam_n lam_n'
// Point values for the upwind convection of Section 4.1 (its facet switch is
// pointwise, so the device evaluates it at fixed nodes):
//   R9[q][i][a]  = phi_{i,a}(x_q)                  R10[q][i][a][b] = d_b phi_{i,a}(x_q)
//   R11[q][n]    = lam_n(x_q)                      R12[q] = weight of node x_q
//   R13[f][g][i][a] = phi_{i,a}(x_f(s_g))          R14[f][g][n] = lam_n(x_f(s_g))
//   R15[g][m]    = l_m(s_g)                        R16[g] = weight of s_g on [0,1]
// with the volume nodes of the Duffy rule above and nfq = (3k+5)/2 Gauss-Legendre
// nodes s_g per facet (exact for the facet terms away from a switch, degree 3k+3).
#include <algorithm>
#include <array>
#include <cmath>
#include <stdexcept>
#include <vector>

#include "hdg_internal.h"

namespace hdg {
namespace {

// polynomial in (x, y) of total degree <= deg, coefficient of x^a y^b at idx(a, b)
struct Poly {
    int deg = 0;
    std::vector<double> c;
    explicit Poly(int d = 0) : deg(d), c((d + 1) * (d + 2) / 2, 0.0) {}
    static int idx(int a, int b) { int n = a + b; return n * (n + 1) / 2 + b; }
    double &at(int a, int b) { return c[idx(a, b)]; }
    double get(int a, int b) const {
        return (a + b <= deg && a >= 0 && b >= 0) ? c[idx(a, b)] : 0.0;
    }
};

Poly mul(const Poly &p, const Poly &q) {
    Poly r(p.deg + q.deg);
    for (int n = 0; n <= p.deg; ++n)
        for (int b = 0; b <= n; ++b) {
            double pc = p.c[Poly::idx(n - b, b)];
            if (pc == 0.0) continue;
            for (int m = 0; m <= q.deg; ++m)
                for (int d = 0; d <= m; ++d)
                    r.at(n - b + m - d, b + d) += pc * q.c[Poly::idx(m - d, d)];
        }
    return r;
}

Poly add(const Poly &p, const Poly &q, double s = 1.0) {
    Poly r(std::max(p.deg, q.deg));
    for (int n = 0; n <= r.deg; ++n)
        for (int b = 0; b <= n; ++b) r.at(n - b, b) = p.get(n - b, b) + s * q.get(n - b, b);
    return r;
}

Poly scale(const Poly &p, double s) {
    Poly r = p;
    for (double &v : r.c) v *= s;
    return r;
}

Poly deriv(const Poly &p, int dir) {
    Poly r(std::max(p.deg - 1, 0));
    for (int n = 1; n <= p.deg; ++n)
        for (int b = 0; b <= n; ++b) {
            int a = n - b;
            double v = p.c[Poly::idx(a, b)];
            if (dir == 0 && a > 0) r.at(a - 1, b) += a * v;
            if (dir == 1 && b > 0) r.at(a, b - 1) += b * v;
        }
    return r;
}

double fact(int n) { double r = 1; for (int i = 2; i <= n; ++i) r *= i; return r; }

double integrate(const Poly &p) {
    double s = 0;
    for (int n = 0; n <= p.deg; ++n)
        for (int b = 0; b <= n; ++b) {
            int a = n - b;
            s += p.c[Poly::idx(a, b)] * fact(a) * fact(b) / fact(a + b + 2);
        }
    return s;
}

Poly monomial(int a, int b) { Poly p(a + b); p.at(a, b) = 1.0; return p; }

// 1D polynomial in s (coefficients of s^i)
using Poly1 = std::vector<double>;

Poly1 mul1(const Poly1 &p, const Poly1 &q) {
    Poly1 r(p.size() + q.size() - 1, 0.0);
    for (size_t i = 0; i < p.size(); ++i)
        for (size_t j = 0; j < q.size(); ++j) r[i + j] += p[i] * q[j];
    return r;
}

double integrate1(const Poly1 &p) {
    double s = 0;
    for (size_t i = 0; i < p.size(); ++i) s += p[i] / double(i + 1);
    return s;
}

// restriction of p to x(s) = X0 + s (X1 - X0)
Poly1 restrict_to(const Poly &p, const double X0[2], const double X1[2]) {
    Poly1 r(p.deg + 1, 0.0);
    Poly1 px = {X0[0], X1[0] - X0[0]}, py = {X0[1], X1[1] - X0[1]};
    for (int n = 0; n <= p.deg; ++n)
        for (int b = 0; b <= n; ++b) {
            int a = n - b;
            double v = p.c[Poly::idx(a, b)];
            if (v == 0.0) continue;
            Poly1 t = {1.0};
            for (int i = 0; i < a; ++i) t = mul1(t, px);
            for (int i = 0; i < b; ++i) t = mul1(t, py);
            for (size_t i = 0; i < t.size(); ++i) r[i] += v * t[i];
        }
    return r;
}

// sqrt(2m+1) P_m(2s-1) as a polynomial in s (three-term recurrence)
Poly1 legendre01(int m) {
    Poly1 P0 = {1.0}, P1 = {-1.0, 2.0};
    if (m == 0) return P0;
    Poly1 a = P0, b = P1;
    for (int n = 1; n < m; ++n) {
        Poly1 tb = mul1(Poly1{-1.0, 2.0}, b);
        Poly1 c(std::max(tb.size(), a.size()), 0.0);
        for (size_t i = 0; i < tb.size(); ++i) c[i] += (2.0 * n + 1) / (n + 1) * tb[i];
        for (size_t i = 0; i < a.size(); ++i) c[i] -= double(n) / (n + 1) * a[i];
        a = b;
        b = c;
    }
    for (double &v : b) v *= std::sqrt(2.0 * m + 1.0);
    return b;
}

// dense inverse by Gauss-Jordan with partial pivoting
std::vector<double> invert(std::vector<double> A, int n) {
    std::vector<double> I(n * n, 0.0);
    for (int i = 0; i < n; ++i) I[i * n + i] = 1.0;
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(A[r * n + c]) > std::fabs(A[p * n + c])) p = r;
        if (std::fabs(A[p * n + c]) < 1e-300) throw std::runtime_error("singular reference matrix");
        for (int j = 0; j < n; ++j) {
            std::swap(A[c * n + j], A[p * n + j]);
            std::swap(I[c * n + j], I[p * n + j]);
        }
        double d = A[c * n + c];
        for (int j = 0; j < n; ++j) { A[c * n + j] /= d; I[c * n + j] /= d; }
        for (int r = 0; r < n; ++r)
            if (r != c) {
                double f = A[r * n + c];
                if (f == 0.0) continue;
                for (int j = 0; j < n; ++j) {
                    A[r * n + j] -= f * A[c * n + j];
                    I[r * n + j] -= f * I[c * n + j];
                }
            }
    }
    return I;
}

const double RV[3][2] = {{0, 0}, {1, 0}, {0, 1}};
const int FV[3][2] = {{1, 2}, {0, 2}, {0, 1}};        // local vertices of facet f, increasing

} // namespace

// Gauss-Legendre nodes/weights on [0,1] by Newton iteration on P_n
static void gauss_legendre01(int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    const double PI = 3.14159265358979323846;
    for (int i = 0; i < n; ++i) {
        double z = std::cos(PI * (i + 0.75) / (n + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int m = 2; m <= n; ++m) {
                double p2 = ((2.0 * m - 1) * z * p1 - (m - 1.0) * p0) / m;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        // recompute derivative at the converged node
        double p0 = 1.0, p1 = z;
        for (int m = 2; m <= n; ++m) {
            double p2 = ((2.0 * m - 1) * z * p1 - (m - 1.0) * p0) / m;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = 0.5 * (1.0 - z);
        w[i] = 1.0 / ((1.0 - z * z) * dp * dp);   // 2/((1-z^2)P'^2) scaled by 1/2
    }
}

// value and gradient of the centred monomial (x-1/3)^a (y-1/3)^b
static void mono_eval(int a, int b, double x, double y, double &v, double &dx, double &dy) {
    double X = x - 1.0 / 3.0, Y = y - 1.0 / 3.0;
    v = std::pow(X, a) * std::pow(Y, b);
    dx = a > 0 ? a * std::pow(X, a - 1) * std::pow(Y, b) : 0.0;
    dy = b > 0 ? b * std::pow(X, a) * std::pow(Y, b - 1) : 0.0;
}

void build_reference_tables(int k, RefTables &t) {
    t.k = k;
    const int npk = (k + 1) * (k + 2) / 2;
    const int nrt = (k + 1) * (k + 3);
    const int nf = k + 1;
    const int q = k + 1;
    const int nlat = (q + 1) * (q + 2) / 2;
    const int nint = k * (k + 1) / 2;            // dim P^{k-1}
    t.npk = npk; t.nrt = nrt; t.nf = nf; t.nlat = nlat;

    // Duffy rule on the reference triangle: x = u, y = v (1 - u) ... use
    // x = s1, y = s2 (1 - s1), Jacobian (1 - s1), n nodes per direction
    const int n = k + 5;
    std::vector<double> gx, gw;
    gauss_legendre01(n, gx, gw);
    std::vector<double> QX, QY, QW;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            QX.push_back(gx[i]);
            QY.push_back(gx[j] * (1.0 - gx[i]));
            QW.push_back(gw[i] * gw[j] * (1.0 - gx[i]));
        }
    const int nq = (int)QW.size();
    // centred monomials up to degree k+1 at the volume nodes
    std::vector<std::pair<int, int>> ex;
    for (int d = 0; d <= k + 1; ++d)
        for (int b = 0; b <= d; ++b) ex.push_back({d - b, b});
    const int nm = (int)ex.size();
    auto mono_at = [&](double x, double y, std::vector<double> &v, std::vector<double> &dx,
                       std::vector<double> &dy) {
        v.resize(nm); dx.resize(nm); dy.resize(nm);
        for (int m = 0; m < nm; ++m) mono_eval(ex[m].first, ex[m].second, x, y, v[m], dx[m], dy[m]);
    };
    // orthonormal P^k: coefficients over the first npk monomials, Gram-Schmidt (twice)
    std::vector<std::vector<double>> MV(nq), MDX(nq), MDY(nq);
    for (int p = 0; p < nq; ++p) mono_at(QX[p], QY[p], MV[p], MDX[p], MDY[p]);
    auto ip = [&](const std::vector<double> &a, const std::vector<double> &b) {
        double s = 0;
        for (int p = 0; p < nq; ++p) {
            double va = 0, vb = 0;
            for (size_t m = 0; m < a.size(); ++m) va += a[m] * MV[p][m];
            for (size_t m = 0; m < b.size(); ++m) vb += b[m] * MV[p][m];
            s += QW[p] * va * vb;
        }
        return s;
    };
    std::vector<std::vector<double>> G;        // coefficients (length npk)
    for (int i = 0; i < npk; ++i) {
        std::vector<double> v(npk, 0.0);
        v[i] = 1.0;
        for (int pass = 0; pass < 2; ++pass)
            for (const auto &w : G) {
                double c = ip(v, w);
                for (int m = 0; m < npk; ++m) v[m] -= c * w[m];
            }
        double nn = std::sqrt(ip(v, v));
        for (double &c : v) c /= nn;
        G.push_back(v);
    }
    auto g_at = [&](int j, const std::vector<double> &mv) {
        double s = 0;
        for (int m = 0; m < npk; ++m) s += G[j][m] * mv[m];
        return s;
    };
    // RT_k spanning set over centred monomials: (m,0), (0,m), m in P^k; (X h, Y h), h homogeneous deg k
    // stored as coefficient pairs over the nm monomials (degree <= k+1)
    auto mindex = [&](int a, int b) { int d = a + b; return d * (d + 1) / 2 + b; };
    std::vector<std::array<std::vector<double>, 2>> span;
    for (int m = 0; m < npk; ++m) {
        std::array<std::vector<double>, 2> s1{std::vector<double>(nm, 0.0), std::vector<double>(nm, 0.0)};
        s1[0][m] = 1.0;
        span.push_back(s1);
        std::array<std::vector<double>, 2> s2{std::vector<double>(nm, 0.0), std::vector<double>(nm, 0.0)};
        s2[1][m] = 1.0;
        span.push_back(s2);
    }
    for (int b = 0; b <= k; ++b) {
        std::array<std::vector<double>, 2> s3{std::vector<double>(nm, 0.0), std::vector<double>(nm, 0.0)};
        s3[0][mindex(k - b + 1, b)] = 1.0;
        s3[1][mindex(k - b, b + 1)] = 1.0;
        span.push_back(s3);
    }
    if ((int)span.size() != nrt) throw std::runtime_error("RT span size");
    auto eval_vec = [&](const std::array<std::vector<double>, 2> &f, const std::vector<double> &mv, int a) {
        double s = 0;
        for (int m = 0; m < nm; ++m) s += f[a][m] * mv[m];
        return s;
    };
    // facet nodes (Gauss-Legendre in s, n points)
    const double FVX[3][2][2] = {{{1, 0}, {0, 1}}, {{0, 0}, {0, 1}}, {{0, 0}, {1, 0}}};
    const double fl[3] = {std::sqrt(2.0), 1.0, 1.0};
    const double fn[3][2] = {{1 / std::sqrt(2.0), 1 / std::sqrt(2.0)}, {-1, 0}, {0, -1}};
    auto leg = [&](int m, double s) {
        double z = 2 * s - 1, p0 = 1.0, p1 = z;
        if (m == 0) return 1.0;
        for (int i = 2; i <= m; ++i) {
            double p2 = ((2.0 * i - 1) * z * p1 - (i - 1.0) * p0) / i;
            p0 = p1;
            p1 = p2;
        }
        return std::sqrt(2.0 * m + 1) * p1;
    };
    // DOF matrix V[dof][span]
    std::vector<double> V(nrt * nrt, 0.0);
    std::vector<double> mv, mdx, mdy;
    for (int j = 0; j < nrt; ++j) {
        int row = 0;
        for (int f = 0; f < 3; ++f)
            for (int m = 0; m < nf; ++m, ++row) {
                double s = 0;
                for (int p = 0; p < n; ++p) {
                    double x = FVX[f][0][0] + gx[p] * (FVX[f][1][0] - FVX[f][0][0]);
                    double y = FVX[f][0][1] + gx[p] * (FVX[f][1][1] - FVX[f][0][1]);
                    mono_at(x, y, mv, mdx, mdy);
                    double vn = fn[f][0] * eval_vec(span[j], mv, 0) + fn[f][1] * eval_vec(span[j], mv, 1);
                    s += gw[p] * fl[f] * vn * leg(m, gx[p]);
                }
                V[row * nrt + j] = s;
            }
        for (int a = 0; a < 2; ++a)
            for (int r = 0; r < nint; ++r, ++row) {
                double s = 0;
                for (int p = 0; p < nq; ++p) s += QW[p] * eval_vec(span[j], MV[p], a) * g_at(r, MV[p]);
                V[row * nrt + j] = s;
            }
    }
    std::vector<double> Vi = invert(V, nrt);
    // dual basis phi_i = sum_j span_j Vi[j][i] (coefficients over monomials)
    std::vector<std::array<std::vector<double>, 2>> phi(nrt, {std::vector<double>(nm, 0.0), std::vector<double>(nm, 0.0)});
    for (int i = 0; i < nrt; ++i)
        for (int j = 0; j < nrt; ++j)
            for (int a = 0; a < 2; ++a)
                for (int m = 0; m < nm; ++m) phi[i][a][m] += span[j][a][m] * Vi[j * nrt + i];
    auto phi_val = [&](int i, int a, const std::vector<double> &mvv) { return eval_vec(phi[i], mvv, a); };
    auto phi_der = [&](int i, int a, int b, const std::vector<double> &dxx, const std::vector<double> &dyy) {
        const std::vector<double> &d = b == 0 ? dxx : dyy;
        double s = 0;
        for (int m = 0; m < nm; ++m) s += phi[i][a][m] * d[m];
        return s;
    };
    // Lagrange basis of P^q on the lattice: Vandermonde over centred monomials (degree q = k+1 = nm set)
    std::vector<double> Lv(nlat * nlat, 0.0);
    {
        int pidx = 0;
        for (int a2 = 0; a2 <= q; ++a2)
            for (int a1 = 0; a1 <= q - a2; ++a1, ++pidx) {
                mono_at(double(a1) / q, double(a2) / q, mv, mdx, mdy);
                for (int c = 0; c < nlat; ++c) Lv[pidx * nlat + c] = mv[c];
            }
    }
    std::vector<double> Li = invert(Lv, nlat);
    auto lam_val = [&](int nn, const std::vector<double> &mvv) {
        double s = 0;
        for (int c = 0; c < nlat; ++c) s += Li[c * nlat + nn] * mvv[c];
        return s;
    };

    t.R1.assign((size_t)nrt * 4 * npk, 0.0);
    t.R2.assign((size_t)3 * nrt * 2 * npk, 0.0);
    t.R3.assign((size_t)3 * npk * nf, 0.0);
    t.R4.assign((size_t)nrt * 2 * nrt * 2, 0.0);
    t.R5.assign((size_t)nrt * npk, 0.0);
    t.R6.assign((size_t)nrt * 2 * nlat, 0.0);
    t.R7.assign((size_t)nrt * 2 * nlat, 0.0);
    t.R8.assign((size_t)nlat * nlat, 0.0);
    const int nfq = (3 * k + 5) / 2;
    t.nq = nq;
    t.nfq = nfq;
    t.R9.assign((size_t)nq * nrt * 2, 0.0);
    t.R10.assign((size_t)nq * nrt * 4, 0.0);
    t.R11.assign((size_t)nq * nlat, 0.0);
    t.R12.assign((size_t)nq, 0.0);
    t.R13.assign((size_t)3 * nfq * nrt * 2, 0.0);
    t.R14.assign((size_t)3 * nfq * nlat, 0.0);
    t.R15.assign((size_t)nfq * nf, 0.0);
    t.R16.assign((size_t)nfq, 0.0);
    t.P1.assign((size_t)4 * nlat * nlat, 0.0);
    t.P2.assign((size_t)npk * nlat * 2, 0.0);
    t.P3.assign((size_t)nlat, 0.0);
    {
        int pidx = 0;
        for (int a2 = 0; a2 <= q; ++a2)
            for (int a1 = 0; a1 <= q - a2; ++a1, ++pidx) {
                mono_at(double(a1) / q, double(a2) / q, mv, mdx, mdy);
                for (int i = 0; i < nrt; ++i)
                    for (int a = 0; a < 2; ++a) t.R7[(i * 2 + a) * nlat + pidx] = phi_val(i, a, mv);
            }
    }
    for (int p = 0; p < nq; ++p) {
        const auto &mvp = MV[p], &dxp = MDX[p], &dyp = MDY[p];
        std::vector<double> gv(npk), lv(nlat), pv(nrt * 2), dv(nrt * 4);
        for (int j = 0; j < npk; ++j) gv[j] = g_at(j, mvp);
        for (int nn = 0; nn < nlat; ++nn) lv[nn] = lam_val(nn, mvp);
        for (int i = 0; i < nrt; ++i)
            for (int a = 0; a < 2; ++a) {
                pv[2 * i + a] = phi_val(i, a, mvp);
                for (int b = 0; b < 2; ++b) dv[(2 * i + a) * 2 + b] = phi_der(i, a, b, dxp, dyp);
            }
        const double wq = QW[p];
        for (int i = 0; i < nrt; ++i)
            for (int a = 0; a < 2; ++a) {
                t.R9[((size_t)p * nrt + i) * 2 + a] = pv[2 * i + a];
                for (int b = 0; b < 2; ++b) t.R10[(((size_t)p * nrt + i) * 2 + a) * 2 + b] = dv[(2 * i + a) * 2 + b];
            }
        for (int nn = 0; nn < nlat; ++nn) t.R11[(size_t)p * nlat + nn] = lv[nn];
        t.R12[p] = wq;
        for (int i = 0; i < nrt; ++i) {
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b)
                    for (int j = 0; j < npk; ++j)
                        t.R1[((i * 2 + a) * 2 + b) * npk + j] += wq * dv[(2 * i + a) * 2 + b] * gv[j];
            for (int a = 0; a < 2; ++a)
                for (int i2 = 0; i2 < nrt; ++i2)
                    for (int b = 0; b < 2; ++b)
                        t.R4[((i * 2 + a) * nrt + i2) * 2 + b] += wq * pv[2 * i + a] * pv[2 * i2 + b];
            double div = dv[(2 * i) * 2 + 0] + dv[(2 * i + 1) * 2 + 1];
            for (int j = 0; j < npk; ++j) t.R5[i * npk + j] += wq * div * gv[j];
            for (int a = 0; a < 2; ++a)
                for (int nn = 0; nn < nlat; ++nn) t.R6[(i * 2 + a) * nlat + nn] += wq * pv[2 * i + a] * lv[nn];
        }
        for (int n1 = 0; n1 < nlat; ++n1)
            for (int n2 = 0; n2 < nlat; ++n2) t.R8[n1 * nlat + n2] += wq * lv[n1] * lv[n2];
        // gradients of the lattice Lagrange basis for the post-processing tables
        std::vector<double> ld(nlat * 2, 0.0);
        for (int nn = 0; nn < nlat; ++nn)
            for (int c = 0; c < nlat; ++c) {
                ld[nn * 2 + 0] += Li[c * nlat + nn] * dxp[c];
                ld[nn * 2 + 1] += Li[c * nlat + nn] * dyp[c];
            }
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                for (int n1 = 0; n1 < nlat; ++n1)
                    for (int n2 = 0; n2 < nlat; ++n2)
                        t.P1[((size_t)(a * 2 + b) * nlat + n1) * nlat + n2] += wq * ld[n1 * 2 + a] * ld[n2 * 2 + b];
        for (int j = 0; j < npk; ++j)
            for (int nn = 0; nn < nlat; ++nn)
                for (int b = 0; b < 2; ++b) t.P2[((size_t)j * nlat + nn) * 2 + b] += wq * gv[j] * ld[nn * 2 + b];
        for (int nn = 0; nn < nlat; ++nn) t.P3[nn] += wq * lv[nn];
    }
    for (int f = 0; f < 3; ++f)
        for (int p = 0; p < n; ++p) {
            double x = FVX[f][0][0] + gx[p] * (FVX[f][1][0] - FVX[f][0][0]);
            double y = FVX[f][0][1] + gx[p] * (FVX[f][1][1] - FVX[f][0][1]);
            mono_at(x, y, mv, mdx, mdy);
            for (int j = 0; j < npk; ++j) {
                double gj = g_at(j, mv);
                for (int i = 0; i < nrt; ++i)
                    for (int a = 0; a < 2; ++a)
                        t.R2[((f * nrt + i) * 2 + a) * npk + j] += gw[p] * fl[f] * phi_val(i, a, mv) * gj;
                for (int m = 0; m < nf; ++m) t.R3[(f * npk + j) * nf + m] += gw[p] * gj * leg(m, gx[p]);
            }
        }
    {
        std::vector<double> fx, fw;
        gauss_legendre01(nfq, fx, fw);
        for (int g = 0; g < nfq; ++g) {
            t.R16[g] = fw[g];
            for (int m = 0; m < nf; ++m) t.R15[g * nf + m] = leg(m, fx[g]);
            for (int f = 0; f < 3; ++f) {
                double x = FVX[f][0][0] + fx[g] * (FVX[f][1][0] - FVX[f][0][0]);
                double y = FVX[f][0][1] + fx[g] * (FVX[f][1][1] - FVX[f][0][1]);
                mono_at(x, y, mv, mdx, mdy);
                for (int i = 0; i < nrt; ++i)
                    for (int a = 0; a < 2; ++a)
                        t.R13[(((size_t)f * nfq + g) * nrt + i) * 2 + a] = phi_val(i, a, mv);
                for (int nn = 0; nn < nlat; ++nn) t.R14[((size_t)f * nfq + g) * nlat + nn] = lam_val(nn, mv);
            }
        }
    }
}

const std::vector<double> *ref_table(const RefTables &t, int which) {
    const std::vector<double> *tabs[16] = {&t.R1,  &t.R2,  &t.R3,  &t.R4,  &t.R5,  &t.R6,  &t.R7,  &t.R8,
                                           &t.R9,  &t.R10, &t.R11, &t.R12, &t.R13, &t.R14, &t.R15, &t.R16};
    return tabs[which];
}

size_t ref_table_offset(const RefTables &t, int which) {
    size_t off = 0;
    for (int i = 0; i < which; ++i) off += ref_table(t, i)->size();
    return off;
}

} // namespace hdg
