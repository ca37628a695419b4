// Host topology of tetrahedral levels: faces, edges, edge patches and their colouring, and
// the transfer slots between a coarse level and its red refinement (Sections 2, 3.4.2).
//
// Conventions (they fix the layout of every 3D skeleton vector):
//  * a face is its sorted global vertex triple; faces are numbered in lexicographic order;
//    local face f of a cell is the face opposite local vertex f; interior faces own the
//    unknowns, numbered in increasing face id;
//  * an edge is its sorted vertex pair, numbered lexicographically; edges are coloured
//    greedily in id order so that two edges of one colour never lie in a common cell, and
//    the edge patch of e holds the interior faces containing e (block smoother of Section
//    3.4.2 with edges in place of vertices);
//  * the face frame and basis follow the sorted vertex order (kernels compute them).
#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <string>
#include <vector>

#include "hdg3d_internal.h"

namespace hdg {
namespace {

const int FV[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
const int EV[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

struct FaceKey {
    int32_t v[3];
    int32_t cell, lf;
};

bool key_less(const FaceKey &a, const FaceKey &b) {
    if (a.v[0] != b.v[0]) return a.v[0] < b.v[0];
    if (a.v[1] != b.v[1]) return a.v[1] < b.v[1];
    if (a.v[2] != b.v[2]) return a.v[2] < b.v[2];
    return a.cell < b.cell;
}

// barycentric coordinates of x in the tetrahedron with vertices X[4][3]
std::array<double, 4> bary(const double X[4][3], const double x[3]) {
    double J[3][3], r[3];
    for (int i = 0; i < 3; ++i) {
        for (int a = 0; a < 3; ++a) J[i][a] = X[a + 1][i] - X[0][i];
        r[i] = x[i] - X[0][i];
    }
    const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                       J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                       J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    double l[3];
    for (int a = 0; a < 3; ++a) {
        double M[3][3];
        for (int i = 0; i < 3; ++i)
            for (int b = 0; b < 3; ++b) M[i][b] = b == a ? r[i] : J[i][b];
        l[a] = (M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0])) / det;
    }
    return {1.0 - l[0] - l[1] - l[2], l[0], l[1], l[2]};
}

// frame (n, t1, t2) and area of the face with sorted vertices a < b < c
void face_frame(const std::vector<double> &X, const int32_t *v, double n[3], double t1[3], double t2[3],
                double &area) {
    double e1[3], e2[3];
    for (int d = 0; d < 3; ++d) {
        e1[d] = X[3 * (size_t)v[1] + d] - X[3 * (size_t)v[0] + d];
        e2[d] = X[3 * (size_t)v[2] + d] - X[3 * (size_t)v[0] + d];
    }
    double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    const double nc = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    const double ne = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    for (int d = 0; d < 3; ++d) {
        n[d] = cr[d] / nc;
        t1[d] = e1[d] / ne;
    }
    t2[0] = n[1] * t1[2] - n[2] * t1[1];
    t2[1] = n[2] * t1[0] - n[0] * t1[2];
    t2[2] = n[0] * t1[1] - n[1] * t1[0];
    area = 0.5 * nc;
}

} // namespace

std::string build_level_topology_3d(HostLevel3 &L) {
    const int64_t nc = L.nc;
    for (int64_t c = 0; c < nc; ++c)
        for (int v = 0; v < 4; ++v) {
            const int32_t g = L.cells[4 * c + v];
            if (g < 0 || g >= L.nv) return "cell vertex index out of range";
            for (int w = 0; w < v; ++w)
                if (L.cells[4 * c + w] == g) return "repeated vertex in a cell";
        }
    // faces
    std::vector<FaceKey> keys((size_t)4 * nc);
    for (int64_t c = 0; c < nc; ++c)
        for (int f = 0; f < 4; ++f) {
            FaceKey &k = keys[4 * c + f];
            for (int i = 0; i < 3; ++i) k.v[i] = L.cells[4 * c + FV[f][i]];
            std::sort(k.v, k.v + 3);
            k.cell = (int32_t)c;
            k.lf = f;
        }
    std::sort(keys.begin(), keys.end(), key_less);
    L.cell_face.assign(4 * nc, -1);
    L.face_v.clear();
    L.face_cells.clear();
    L.face_lf.clear();
    int64_t nf = 0;
    for (size_t i = 0; i < keys.size();) {
        size_t j = i + 1;
        while (j < keys.size() && keys[j].v[0] == keys[i].v[0] && keys[j].v[1] == keys[i].v[1] &&
               keys[j].v[2] == keys[i].v[2])
            ++j;
        if (j - i > 2) return "non-manifold face";
        for (int q = 0; q < 3; ++q) L.face_v.push_back(keys[i].v[q]);
        for (size_t q = 0; q < 2; ++q) {
            L.face_cells.push_back(i + q < j ? keys[i + q].cell : -1);
            L.face_lf.push_back(i + q < j ? keys[i + q].lf : -1);
        }
        for (size_t q = i; q < j; ++q) L.cell_face[4 * (size_t)keys[q].cell + keys[q].lf] = (int32_t)nf;
        ++nf;
        i = j;
    }
    L.nf = nf;
    L.interior_index.assign(nf, -1);
    L.interior_faces.clear();
    for (int64_t F = 0; F < nf; ++F)
        if (L.face_cells[2 * F + 1] >= 0) {
            L.interior_index[F] = (int32_t)L.interior_faces.size();
            L.interior_faces.push_back((int32_t)F);
        }
    L.n_int = (int64_t)L.interior_faces.size();
    // edges
    std::vector<std::array<int32_t, 3>> ek((size_t)6 * nc);
    for (int64_t c = 0; c < nc; ++c)
        for (int e = 0; e < 6; ++e) {
            int32_t a = L.cells[4 * c + EV[e][0]], b = L.cells[4 * c + EV[e][1]];
            ek[6 * c + e] = {std::min(a, b), std::max(a, b), (int32_t)(6 * c + e)};
        }
    std::sort(ek.begin(), ek.end());
    std::vector<int32_t> cell_edge((size_t)6 * nc);
    L.edge_v.clear();
    int64_t ne = 0;
    for (size_t i = 0; i < ek.size();) {
        size_t j = i;
        while (j < ek.size() && ek[j][0] == ek[i][0] && ek[j][1] == ek[i][1]) {
            cell_edge[ek[j][2]] = (int32_t)ne;
            ++j;
        }
        L.edge_v.push_back(ek[i][0]);
        L.edge_v.push_back(ek[i][1]);
        ++ne;
        i = j;
    }
    L.ne = ne;
    std::vector<std::vector<int32_t>> ecells(ne);
    for (int64_t c = 0; c < nc; ++c)
        for (int e = 0; e < 6; ++e) ecells[cell_edge[6 * c + e]].push_back((int32_t)c);
    // greedy colouring: edges sharing a cell differ
    L.colour.assign(ne, -1);
    int ncol = 0;
    std::vector<int> mark;
    for (int64_t e = 0; e < ne; ++e) {
        for (int32_t c : ecells[e])
            for (int q = 0; q < 6; ++q) {
                const int32_t col = L.colour[cell_edge[6 * (size_t)c + q]];
                if (col >= 0) {
                    if ((int)mark.size() <= col) mark.resize(col + 1, -1);
                    mark[col] = (int)e;
                }
            }
        int col = 0;
        while (col < (int)mark.size() && mark[col] == (int)e) ++col;
        L.colour[e] = col;
        ncol = std::max(ncol, col + 1);
    }
    // patches: interior faces containing each edge
    std::map<std::pair<int32_t, int32_t>, int32_t> eid;
    for (int64_t e = 0; e < ne; ++e) eid[{L.edge_v[2 * e], L.edge_v[2 * e + 1]}] = (int32_t)e;
    std::vector<std::vector<int32_t>> inc(ne);
    for (int64_t i = 0; i < L.n_int; ++i) {
        const int32_t *v = &L.face_v[3 * (size_t)L.interior_faces[i]];
        inc[eid[{v[0], v[1]}]].push_back((int32_t)i);
        inc[eid[{v[0], v[2]}]].push_back((int32_t)i);
        inc[eid[{v[1], v[2]}]].push_back((int32_t)i);
    }
    std::vector<int32_t> order;
    for (int64_t e = 0; e < ne; ++e)
        if (!inc[e].empty()) order.push_back((int32_t)e);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return L.colour[a] < L.colour[b]; });
    L.n_patches = (int)order.size();
    L.n_colours = ncol;
    L.pf_max = L.pc_max = 0;
    for (int32_t e : order) {
        L.pf_max = std::max<int>(L.pf_max, (int)inc[e].size());
        L.pc_max = std::max<int>(L.pc_max, (int)ecells[e].size());
    }
    if (L.pc_max > 64) return "an edge lies in more than 64 cells";
    L.colour_ptr.assign(ncol + 1, 0);
    for (int32_t e : order) L.colour_ptr[L.colour[e] + 1]++;
    for (int c = 0; c < ncol; ++c) L.colour_ptr[c + 1] += L.colour_ptr[c];
    const int pf = L.pf_max, pc = L.pc_max;
    L.patch_nf.assign(L.n_patches, 0);
    L.patch_facets.assign((size_t)L.n_patches * pf, -1);
    L.patch_nc.assign(L.n_patches, 0);
    L.patch_cells.assign((size_t)L.n_patches * pc, -1);
    L.patch_slot_src.assign((size_t)L.n_patches * pf * 2, -1);
    L.patch_cext.assign((size_t)L.n_patches * pc * 2, -1);
    for (int p = 0; p < L.n_patches; ++p) {
        const int32_t e = order[p];
        std::vector<int32_t> fac = inc[e], cl = ecells[e];
        std::sort(fac.begin(), fac.end());
        std::sort(cl.begin(), cl.end());
        L.patch_nf[p] = (int)fac.size();
        L.patch_nc[p] = (int)cl.size();
        for (size_t s = 0; s < cl.size(); ++s) {
            L.patch_cells[(size_t)p * pc + s] = cl[s];
            // face f lies opposite local vertex f: the two faces without the edge are those
            // opposite its end points
            int w = 0;
            for (int f = 0; f < 4; ++f) {
                const int32_t vf = L.cells[4 * (size_t)cl[s] + f];
                if (vf == L.edge_v[2 * (size_t)e] || vf == L.edge_v[2 * (size_t)e + 1]) {
                    if (w == 2) return "edge star inconsistent";
                    L.patch_cext[((size_t)p * pc + s) * 2 + w++] = f;
                }
            }
            if (w != 2) return "edge star inconsistent";
        }
        for (size_t j = 0; j < fac.size(); ++j) {
            L.patch_facets[(size_t)p * pf + j] = fac[j];
            const int32_t F = L.interior_faces[fac[j]];
            for (int q = 0; q < 2; ++q) {
                const int32_t c = L.face_cells[2 * F + q], lf = L.face_lf[2 * F + q];
                const int si = (int)(std::find(cl.begin(), cl.end(), c) - cl.begin());
                if (si >= (int)cl.size()) return "patch face outside its star";
                L.patch_slot_src[((size_t)p * pf + j) * 2 + q] = (si << 2) | lf;
            }
        }
    }
    return "";
}

std::string build_transfer_3d(const HostLevel3 &C, const HostLevel3 &F, HostTransfer3 &T) {
    const int64_t ncc = C.nc;
    T = HostTransfer3();
    T.nc_coarse = ncc;
    std::vector<std::vector<int32_t>> ch(ncc);
    for (int64_t c = 0; c < F.nc; ++c) {
        const int32_t P = F.parent[c];
        if (P < 0 || P >= ncc) return "parent index out of range";
        ch[P].push_back((int32_t)c);
    }
    T.slots.assign((size_t)ncc * TR3_SLOTS, -1);
    T.nbr.assign((size_t)ncc * TR3_B, -1);
    T.children.assign((size_t)ncc * 8, -1);
    T.child_slot.assign((size_t)ncc * 32, -1);
    T.W.assign((size_t)ncc * TR3_B * 36, 0.0);
    // slot of each fine face in each coarse cell: (P, slot) pairs per fine face id
    std::vector<std::array<int32_t, 2>> owner(F.nf, {-1, -1});
    auto add_owner = [&](int32_t face, int32_t code) {
        auto &o = owner[face];
        if (o[0] < 0) o[0] = code;
        else if (o[1] < 0 && o[0] != code) o[1] = code;
    };
    for (int64_t P = 0; P < ncc; ++P) {
        if (ch[P].size() != 8) return "a coarse cell without eight children (red refinement expected)";
        std::sort(ch[P].begin(), ch[P].end());
        double X[4][3];
        for (int v = 0; v < 4; ++v)
            for (int d = 0; d < 3; ++d) X[v][d] = C.coords[3 * (size_t)C.cells[4 * P + v] + d];
        double h = 0.0;
        for (int v = 1; v < 4; ++v)
            for (int d = 0; d < 3; ++d) h = std::max(h, std::fabs(X[v][d] - X[0][d]));
        std::vector<int32_t> onface[4], inner;
        for (int q = 0; q < 8; ++q) {
            const int32_t c = ch[P][q];
            T.children[8 * P + q] = c;
            for (int lf = 0; lf < 4; ++lf) {
                const int32_t Ff = F.cell_face[4 * (size_t)c + lf];
                double m[3] = {0, 0, 0};
                for (int i = 0; i < 3; ++i)
                    for (int d = 0; d < 3; ++d) m[d] += F.coords[3 * (size_t)F.face_v[3 * (size_t)Ff + i] + d] / 3.0;
                auto lam = bary(X, m);
                int cf = -1;
                for (int i = 0; i < 4; ++i)
                    if (std::fabs(lam[i]) < 1e-9) cf = i;
                auto &lst = cf >= 0 ? onface[cf] : inner;
                if (std::find(lst.begin(), lst.end(), Ff) == lst.end()) lst.push_back(Ff);
            }
        }
        std::sort(inner.begin(), inner.end());
        if (inner.size() != TR3_T) return "a coarse cell whose children have " + std::to_string(inner.size()) +
                                          " inner faces (8 expected)";
        std::vector<int32_t> slot_face(TR3_SLOTS, -1);
        for (int cf = 0; cf < 4; ++cf) {
            std::sort(onface[cf].begin(), onface[cf].end());
            if (onface[cf].size() != 4) return "a coarse face not split into four fine faces";
            for (int i = 0; i < 4; ++i) slot_face[4 * cf + i] = onface[cf][i];
        }
        for (int t = 0; t < TR3_T; ++t) slot_face[TR3_B + t] = inner[t];
        for (int s = 0; s < TR3_SLOTS; ++s) {
            const int32_t Ff = slot_face[s];
            T.slots[TR3_SLOTS * P + s] = F.interior_index[Ff];
            if (F.interior_index[Ff] >= 0) add_owner(Ff, (int32_t)((P << 5) | s));
        }
        for (int q = 0; q < 8; ++q)
            for (int lf = 0; lf < 4; ++lf) {
                const int32_t Ff = F.cell_face[4 * (size_t)ch[P][q] + lf];
                if (F.interior_index[Ff] < 0) continue;
                const int s = (int)(std::find(slot_face.begin(), slot_face.end(), Ff) - slot_face.begin());
                T.child_slot[32 * P + 4 * q + lf] = s;
            }
        // averaging weights of the B slots (eq. avgOpt; the two sides' 1/2 included)
        for (int s = 0; s < TR3_B; ++s) {
            const int32_t Ff = slot_face[s];
            if (F.interior_index[Ff] < 0) continue;
            double nf[3], t1f[3], t2f[3], af;
            face_frame(F.coords, &F.face_v[3 * (size_t)Ff], nf, t1f, t2f, af);
            double m[3] = {0, 0, 0};
            for (int i = 0; i < 3; ++i)
                for (int d = 0; d < 3; ++d) m[d] += F.coords[3 * (size_t)F.face_v[3 * (size_t)Ff + i] + d] / 3.0;
            auto lam = bary(X, m);
            const double *ef[3] = {nf, t1f, t2f};
            for (int i = 0; i < 4; ++i) {
                const int32_t Fc = C.cell_face[4 * P + i];
                if (C.interior_index[Fc] < 0) continue;
                double nc[3], t1c[3], t2c[3], ac;
                face_frame(C.coords, &C.face_v[3 * (size_t)Fc], nc, t1c, t2c, ac);
                const double *ec[3] = {nc, t1c, t2c};
                const double psi = 1.0 - 3.0 * lam[i];
                for (int a = 0; a < 3; ++a)
                    for (int a2 = 0; a2 < 3; ++a2) {
                        const double dot = ef[a][0] * ec[a2][0] + ef[a][1] * ec[a2][1] + ef[a][2] * ec[a2][2];
                        T.W[((size_t)P * TR3_B + s) * 36 + a * 12 + 3 * i + a2] =
                            0.5 * std::sqrt(af) * dot * psi / std::sqrt(ac);
                    }
            }
        }
        (void)h;
    }
    // neighbours of B slots and the list of fine faces on coarse interior faces
    for (int64_t Ff = 0; Ff < F.nf; ++Ff) {
        const auto &o = owner[Ff];
        if (o[0] < 0) continue;
        const int s0 = o[0] & 31;
        if (s0 >= TR3_B) continue;           // inside a coarse cell
        if (o[1] < 0) return "a fine face on a coarse interior face with one coarse side";
        T.nbr[(size_t)(o[0] >> 5) * TR3_B + s0] = o[1];
        T.nbr[(size_t)(o[1] >> 5) * TR3_B + (o[1] & 31)] = o[0];
        T.fineB.push_back(F.interior_index[Ff]);
        T.fineB_src.push_back(o[0]);
        T.fineB_src.push_back(o[1]);
    }
    T.nB = (int64_t)T.fineB.size();
    return "";
}

} // namespace hdg
