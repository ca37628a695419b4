// Host-side mesh topology for the H(div)-HDG hierarchy.
//
// * Facets (Section 2): identified by sorted vertex pairs, numbered in
//   lexicographic order; local facet f of a cell is opposite local vertex f;
//   interior facets (two cells) own the skeleton unknowns, boundary facets
//   carry the homogeneous Dirichlet condition (Section 3.1).
// * Vertex patches (Section 3.4.2, subspaces V^{0,s}; Section 3.5): the patch
//   of vertex s holds the interior facets containing s and the cells around s.
//   Patches are ordered by colour of a proper vertex colouring; two vertices
//   of one colour share no cell, so their block updates commute and one
//   colour runs as one parallel phase of block Gauss-Seidel.
// * Transfer maps (eq. avgOpt, eqs. div-transfer/harmonic-ex): for each coarse
//   cell its four children, the six fine facets on its boundary (slots 0..5,
//   two per coarse local facet, the half next to the lower local vertex
//   first) and the three fine facets inside it (slots 6..8), and the weights
//   that evaluate the coarse Crouzeix-Raviart function Π^CR at the midpoints
//   of the boundary fine facets.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <numeric>
#include <tuple>

#include "hdg_internal.h"

namespace hdg {

static void facet_geometry(const HostLevel &L, int F, double xl[2], double &len, double t[2],
                           double n[2]) {
    int a = L.facet_v[2 * F], b = L.facet_v[2 * F + 1];
    xl[0] = L.coords[2 * a];
    xl[1] = L.coords[2 * a + 1];
    double dx = L.coords[2 * b] - xl[0], dy = L.coords[2 * b + 1] - xl[1];
    len = std::sqrt(dx * dx + dy * dy);
    t[0] = dx / len;
    t[1] = dy / len;
    n[0] = t[1];
    n[1] = -t[0];
}

std::string build_level_topology(HostLevel &L, const int32_t *colour_in) {
    const int64_t nc = L.nc, nv = L.nv;
    for (int64_t c = 0; c < nc; ++c)
        for (int i = 0; i < 3; ++i) {
            int v = L.cells[3 * c + i];
            if (v < 0 || v >= nv) return "cell vertex id out of range";
        }
    // facet incidences (min, max, cell, lf)
    std::vector<std::array<int64_t, 4>> inc(3 * nc);
    for (int64_t c = 0; c < nc; ++c)
        for (int f = 0; f < 3; ++f) {
            int a = L.cells[3 * c + (f + 1) % 3], b = L.cells[3 * c + (f + 2) % 3];
            if (a == b) return "degenerate cell";
            inc[3 * c + f] = {std::min(a, b), std::max(a, b), c, f};
        }
    std::sort(inc.begin(), inc.end());
    L.facet_v.clear();
    L.facet_cells.clear();
    L.facet_lf.clear();
    L.cell_facet.assign(3 * nc, -1);
    for (size_t i = 0; i < inc.size();) {
        size_t j = i;
        while (j < inc.size() && inc[j][0] == inc[i][0] && inc[j][1] == inc[i][1]) ++j;
        if (j - i > 2) return "non-manifold facet";
        int F = (int)(L.facet_v.size() / 2);
        L.facet_v.push_back((int32_t)inc[i][0]);
        L.facet_v.push_back((int32_t)inc[i][1]);
        for (size_t q = 0; q < 2; ++q) {
            if (i + q < j) {
                L.facet_cells.push_back((int32_t)inc[i + q][2]);
                L.facet_lf.push_back((int32_t)inc[i + q][3]);
                L.cell_facet[3 * inc[i + q][2] + inc[i + q][3]] = F;
            } else {
                L.facet_cells.push_back(-1);
                L.facet_lf.push_back(-1);
            }
        }
        i = j;
    }
    L.nf = (int64_t)L.facet_v.size() / 2;
    L.interior_index.assign(L.nf, -1);
    L.interior_facets.clear();
    for (int64_t F = 0; F < L.nf; ++F)
        if (L.facet_cells[2 * F + 1] >= 0) {
            L.interior_index[F] = (int32_t)L.interior_facets.size();
            L.interior_facets.push_back((int32_t)F);
        }
    L.n_int = (int64_t)L.interior_facets.size();

    // vertex adjacency via facets
    std::vector<std::vector<int32_t>> vf(nv), vc(nv);
    for (int64_t F = 0; F < L.nf; ++F) {
        vf[L.facet_v[2 * F]].push_back((int32_t)F);
        vf[L.facet_v[2 * F + 1]].push_back((int32_t)F);
    }
    for (int64_t c = 0; c < nc; ++c)
        for (int i = 0; i < 3; ++i) vc[L.cells[3 * c + i]].push_back((int32_t)c);
    // colouring
    L.colour.assign(nv, -1);
    if (colour_in) {
        for (int64_t v = 0; v < nv; ++v) {
            if (colour_in[v] < 0 || colour_in[v] > 255) return "vertex colour out of range";
            L.colour[v] = colour_in[v];
        }
    } else {
        for (int64_t v = 0; v < nv; ++v) {
            std::vector<char> used(vf[v].size() + 2, 0);
            for (int F : vf[v]) {
                int w = L.facet_v[2 * F] == v ? L.facet_v[2 * F + 1] : L.facet_v[2 * F];
                int cw = L.colour[w];
                if (cw >= 0 && cw < (int)used.size()) used[cw] = 1;
            }
            int c = 0;
            while (used[c]) ++c;
            L.colour[v] = c;
        }
    }
    for (int64_t F = 0; F < L.nf; ++F)
        if (L.colour[L.facet_v[2 * F]] == L.colour[L.facet_v[2 * F + 1]])
            return "vertex colouring is not proper";
    int ncol = 0;
    for (int64_t v = 0; v < nv; ++v) ncol = std::max(ncol, L.colour[v] + 1);
    L.n_colours = ncol;

    // patches ordered by (colour, vertex)
    std::vector<int32_t> order(nv);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return L.colour[a] < L.colour[b]; });
    std::vector<std::vector<int32_t>> pf;
    std::vector<int32_t> pv;
    L.pf_max = 0;
    L.pc_max = 0;
    for (int v : order) {
        std::vector<int32_t> fl;
        for (int F : vf[v])
            if (L.interior_index[F] >= 0) fl.push_back(L.interior_index[F]);
        if (fl.empty()) continue;
        std::sort(fl.begin(), fl.end());
        pf.push_back(fl);
        pv.push_back(v);
        L.pf_max = std::max(L.pf_max, (int)fl.size());
        L.pc_max = std::max(L.pc_max, (int)vc[v].size());
    }
    L.n_patches = (int)pv.size();
    L.colour_ptr.assign(ncol + 1, 0);
    for (int p = 0; p < L.n_patches; ++p) L.colour_ptr[L.colour[pv[p]] + 1]++;
    for (int c = 0; c < ncol; ++c) L.colour_ptr[c + 1] += L.colour_ptr[c];
    L.patch_nf.assign(L.n_patches, 0);
    L.patch_nc.assign(L.n_patches, 0);
    L.patch_facets.assign((size_t)L.n_patches * L.pf_max, -1);
    L.patch_cells.assign((size_t)L.n_patches * L.pc_max, -1);
    L.patch_slot_src.assign((size_t)L.n_patches * L.pf_max * 2, -1);
    L.patch_cext.assign((size_t)L.n_patches * L.pc_max, -1);
    for (int p = 0; p < L.n_patches; ++p) {
        int v = pv[p];
        std::vector<int32_t> cs = vc[v];
        std::sort(cs.begin(), cs.end());
        L.patch_nf[p] = (int)pf[p].size();
        L.patch_nc[p] = (int)cs.size();
        for (size_t i = 0; i < cs.size(); ++i) {
            L.patch_cells[(size_t)p * L.pc_max + i] = cs[i];
            // facet f lies opposite local vertex f: the facet of the cell without v
            for (int f = 0; f < 3; ++f)
                if (L.cells[3 * (size_t)cs[i] + f] == v) L.patch_cext[(size_t)p * L.pc_max + i] = f;
            if (L.patch_cext[(size_t)p * L.pc_max + i] < 0) return "patch star inconsistent";
        }
        for (size_t j = 0; j < pf[p].size(); ++j) {
            int F = L.interior_facets[pf[p][j]];
            L.patch_facets[(size_t)p * L.pf_max + j] = pf[p][j];
            for (int q = 0; q < 2; ++q) {
                int c = L.facet_cells[2 * F + q], lf = L.facet_lf[2 * F + q];
                int si = (int)(std::find(cs.begin(), cs.end(), c) - cs.begin());
                if (si >= (int)cs.size()) return "patch star inconsistent";
                L.patch_slot_src[((size_t)p * L.pf_max + j) * 2 + q] = (si << 2) | lf;
            }
        }
    }
    return "";
}

// barycentric coordinates of x in the triangle X (3x2)
static void bary(const double X[6], const double x[2], double lam[3]) {
    double j00 = X[2] - X[0], j01 = X[4] - X[0], j10 = X[3] - X[1], j11 = X[5] - X[1];
    double det = j00 * j11 - j01 * j10;
    double rx = x[0] - X[0], ry = x[1] - X[1];
    lam[1] = (j11 * rx - j01 * ry) / det;
    lam[2] = (-j10 * rx + j00 * ry) / det;
    lam[0] = 1.0 - lam[1] - lam[2];
}

std::string build_transfer(const HostLevel &C, const HostLevel &Fm, HostTransfer &T) {
    const int64_t ncc = C.nc;
    T.nc_coarse = ncc;
    T.children.assign(4 * ncc, -1);
    std::vector<int> cnt(ncc, 0);
    for (int64_t c = 0; c < Fm.nc; ++c) {
        int P = Fm.parent[c];
        if (P < 0 || P >= ncc) return "parent id out of range";
        if (cnt[P] >= 4) return "coarse cell with more than four children";
        T.children[4 * P + cnt[P]++] = (int32_t)c;
    }
    for (int64_t P = 0; P < ncc; ++P)
        if (cnt[P] != 4) return "coarse cell without four children (not a red refinement)";
    T.slots.assign(9 * ncc, -1);
    T.child_slot.assign(12 * ncc, -1);
    T.W.assign(72 * ncc, 0.0);
    std::vector<int32_t> slot_facet(9 * ncc, -1);   // fine facet id per slot
    for (int64_t P = 0; P < ncc; ++P) {
        double X[6];
        for (int i = 0; i < 3; ++i) {
            X[2 * i] = C.coords[2 * C.cells[3 * P + i]];
            X[2 * i + 1] = C.coords[2 * C.cells[3 * P + i] + 1];
        }
        double hmax = 0;
        for (int i = 0; i < 3; ++i) {
            double dx = X[2 * ((i + 1) % 3)] - X[2 * i], dy = X[2 * ((i + 1) % 3) + 1] - X[2 * i + 1];
            hmax = std::max(hmax, std::sqrt(dx * dx + dy * dy));
        }
        std::vector<int32_t> tf;
        int nb = 0;
        for (int ch = 0; ch < 4; ++ch) {
            int c = T.children[4 * P + ch];
            for (int lf = 0; lf < 3; ++lf) {
                int F = Fm.cell_facet[3 * c + lf];
                int c0 = Fm.facet_cells[2 * F], c1 = Fm.facet_cells[2 * F + 1];
                bool inside = c1 >= 0 && Fm.parent[c0] == P && Fm.parent[c1] == P;
                int slot = -1;
                if (inside) {
                    // interior slots assigned after sorting
                    if (std::find(tf.begin(), tf.end(), F) == tf.end()) tf.push_back(F);
                } else {
                    int a = Fm.facet_v[2 * F], b = Fm.facet_v[2 * F + 1];
                    double mid[2] = {0.5 * (Fm.coords[2 * a] + Fm.coords[2 * b]),
                                     0.5 * (Fm.coords[2 * a + 1] + Fm.coords[2 * b + 1])};
                    double lam[3];
                    bary(X, mid, lam);
                    int f = -1;
                    for (int i = 0; i < 3; ++i)
                        if (std::fabs(lam[i]) < 1e-9) f = i;
                    if (f < 0) return "fine boundary facet not on a coarse facet";
                    int la = (f == 0) ? 1 : 0;          // lower local vertex of coarse facet f
                    int lb = (f == 2) ? 1 : 2;
                    slot = 2 * f + (lam[la] > lam[lb] ? 0 : 1);
                    if (slot_facet[9 * P + slot] >= 0 && slot_facet[9 * P + slot] != F)
                        return "two fine facets in one boundary slot";
                    if (slot_facet[9 * P + slot] < 0) nb++;
                    slot_facet[9 * P + slot] = F;
                }
                (void)hmax;
            }
        }
        if (nb != 6 || tf.size() != 3) return "coarse cell is not red-refined";
        std::sort(tf.begin(), tf.end());
        for (int i = 0; i < 3; ++i) slot_facet[9 * P + 6 + i] = tf[i];
        for (int s = 0; s < 9; ++s) T.slots[9 * P + s] = Fm.interior_index[slot_facet[9 * P + s]];
        for (int ch = 0; ch < 4; ++ch) {
            int c = T.children[4 * P + ch];
            for (int lf = 0; lf < 3; ++lf) {
                int F = Fm.cell_facet[3 * c + lf];
                for (int s = 0; s < 9; ++s)
                    if (slot_facet[9 * P + s] == F) T.child_slot[12 * P + 3 * ch + lf] = s;
            }
        }
        // averaging weights: row (slot s, comp r) <- coarse (local facet f', comp q)
        for (int s = 0; s < 6; ++s) {
            int F = slot_facet[9 * P + s];
            double xl[2], lenf, tf2[2], nf2[2];
            facet_geometry(Fm, F, xl, lenf, tf2, nf2);
            int a = Fm.facet_v[2 * F], b = Fm.facet_v[2 * F + 1];
            double mid[2] = {0.5 * (Fm.coords[2 * a] + Fm.coords[2 * b]),
                             0.5 * (Fm.coords[2 * a + 1] + Fm.coords[2 * b + 1])};
            double lam[3];
            bary(X, mid, lam);
            for (int fp = 0; fp < 3; ++fp) {
                int G = C.cell_facet[3 * P + fp];
                double xc[2], lenc, tc[2], nc2[2];
                facet_geometry(C, G, xc, lenc, tc, nc2);
                double psi = 1.0 - 2.0 * lam[fp];
                const double *ef[2] = {nc2, tc};
                const double *er[2] = {nf2, tf2};
                for (int r = 0; r < 2; ++r)
                    for (int q = 0; q < 2; ++q) {
                        double dot = ef[q][0] * er[r][0] + ef[q][1] * er[r][1];
                        T.W[72 * P + (2 * s + r) * 6 + 2 * fp + q] =
                            0.5 * std::sqrt(lenf) * psi * dot / std::sqrt(lenc);
                    }
            }
        }
    }
    // neighbour slots across coarse facets
    T.nbr.assign(6 * ncc, -1);
    for (int64_t P = 0; P < ncc; ++P)
        for (int s = 0; s < 6; ++s) {
            int f = s / 2;
            int G = C.cell_facet[3 * P + f];
            int c0 = C.facet_cells[2 * G], c1 = C.facet_cells[2 * G + 1];
            if (c1 < 0) continue;
            int Q = (c0 == P) ? c1 : c0;
            int F = slot_facet[9 * P + s];
            for (int s2 = 0; s2 < 6; ++s2)
                if (slot_facet[9 * Q + s2] == F) T.nbr[6 * P + s] = (Q << 4) | s2;
            if (T.nbr[6 * P + s] < 0) return "neighbour slot not found";
        }
    // fine interior facets on coarse interior facets
    T.fineB.clear();
    T.fineB_src.clear();
    for (int64_t P = 0; P < ncc; ++P)
        for (int s = 0; s < 6; ++s) {
            int i = T.slots[9 * P + s];
            if (i < 0) continue;
            int nb = T.nbr[6 * P + s];
            int Q = nb >> 4;
            if (Q < P) continue;    // record once, from the lower coarse cell
            T.fineB.push_back(i);
            T.fineB_src.push_back((int32_t)((P << 4) | s));
            T.fineB_src.push_back(nb);
        }
    T.nB = (int64_t)T.fineB.size();
    return "";
}

} // namespace hdg
