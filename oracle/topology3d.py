"""Mesh topology for tetrahedrisations (oracle; test infrastructure only).

Conventions (they fix the layout of every 3D skeleton vector):

* A facet (face) is identified by its sorted global vertex triple (a < b < c);
  faces are numbered in lexicographic order of that triple.  Local face f of a
  cell is the face opposite local vertex f.
* Face frame: t1 = (x_b - x_a)/|x_b - x_a|, n_F = (x_b - x_a) × (x_c - x_a)
  normalised, t2 = n_F × t1.  The face's scalar basis uses the barycentric
  coordinates (λ_b, λ_c) of (x_b, x_c), so both neighbours of a face see the
  same basis.
* Boundary faces (one adjacent cell) carry the Dirichlet condition (Section 3.1)
  and hold no unknowns; interior faces are numbered in increasing face id and
  own the skeleton unknowns.
* Edges are sorted global vertex pairs in lexicographic order.  Edge patches
  (Section 3.4.2: in 3D, patches around edges) are coloured greedily, edges in
  increasing id, so that two edges of one colour never lie in a common cell:
  then no face of one patch lies in a cell of another patch of the same colour,
  and the patches of a colour can be relaxed in any order.
"""

from __future__ import annotations

from dataclasses import dataclass
from typing import List

import numpy as np

LOCAL_EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))


@dataclass
class Topology3D:
    coords: np.ndarray          # (nv, 3)
    cells: np.ndarray           # (nc, 4)
    facets: np.ndarray          # (nf, 3) sorted vertex triples
    cell_facets: np.ndarray     # (nc, 4) face id opposite local vertex f
    facet_cells: np.ndarray     # (nf, 2) adjacent cells (second = -1 on the boundary)
    interior_index: np.ndarray  # (nf,) interior number or -1
    interior_facets: np.ndarray  # (n_int,) face ids of interior faces
    edges: np.ndarray           # (ne, 2) sorted vertex pairs
    cell_edges: np.ndarray      # (nc, 6) edge ids of LOCAL_EDGES
    edge_colour: np.ndarray     # (ne,) greedy colouring (no two edges of a colour share a cell)

    dim = 3

    @property
    def n_cells(self) -> int:
        return int(self.cells.shape[0])

    @property
    def n_interior(self) -> int:
        return int(self.interior_facets.shape[0])

    def facet_geometry(self, F: int):
        """(x_a, x_b, x_c, area, t1, t2, n_F) of face F (vertices in sorted global order)."""
        a, b, c = self.facets[F]
        xa, xb, xc = self.coords[a], self.coords[b], self.coords[c]
        cr = np.cross(xb - xa, xc - xa)
        area = 0.5 * float(np.linalg.norm(cr))
        n = cr / np.linalg.norm(cr)
        t1 = (xb - xa) / np.linalg.norm(xb - xa)
        t2 = np.cross(n, t1)
        return xa, xb, xc, area, t1, t2, n

    def cell_volume(self, c: int) -> float:
        X = self.coords[self.cells[c]]
        return abs(np.linalg.det(np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], axis=1))) / 6.0


def greedy_edge_colouring(n_edges: int, cell_edges: np.ndarray) -> np.ndarray:
    """Smallest-available-colour greedy colouring of the graph 'two edges lie in a common
    cell', edges in increasing id."""
    cells_of = [[] for _ in range(n_edges)]
    for c in range(cell_edges.shape[0]):
        for e in cell_edges[c]:
            cells_of[int(e)].append(c)
    colour = -np.ones(n_edges, dtype=np.int32)
    for e in range(n_edges):
        used = set()
        for c in cells_of[e]:
            for e2 in cell_edges[c]:
                if colour[e2] >= 0:
                    used.add(int(colour[e2]))
        col = 0
        while col in used:
            col += 1
        colour[e] = col
    return colour


def build_topology_3d(coords: np.ndarray, cells: np.ndarray) -> Topology3D:
    cells = np.asarray(cells, dtype=np.int64)
    nc = cells.shape[0]
    keys = {}
    for c in range(nc):
        for f in range(4):
            tri = tuple(sorted(int(cells[c, i]) for i in range(4) if i != f))
            keys.setdefault(tri, []).append((c, f))
    facet_list = sorted(keys.keys())
    fid = {key: i for i, key in enumerate(facet_list)}
    nf = len(facet_list)
    cell_facets = np.empty((nc, 4), dtype=np.int64)
    facet_cells = -np.ones((nf, 2), dtype=np.int64)
    for key, lst in keys.items():
        F = fid[key]
        cs = sorted(c for c, _ in lst)
        if len(cs) > 2:
            raise ValueError("non-manifold face")
        facet_cells[F, :len(cs)] = cs
        for c, f in lst:
            cell_facets[c, f] = F
    interior = facet_cells[:, 1] >= 0
    interior_facets = np.nonzero(interior)[0]
    interior_index = -np.ones(nf, dtype=np.int64)
    interior_index[interior_facets] = np.arange(interior_facets.shape[0])
    ekeys = sorted({tuple(sorted((int(cells[c, a]), int(cells[c, b])))) for c in range(nc)
                    for a, b in LOCAL_EDGES})
    eid = {key: i for i, key in enumerate(ekeys)}
    cell_edges = np.array([[eid[tuple(sorted((int(cells[c, a]), int(cells[c, b]))))]
                            for a, b in LOCAL_EDGES] for c in range(nc)], dtype=np.int64)
    colour = greedy_edge_colouring(len(ekeys), cell_edges)
    return Topology3D(np.asarray(coords, dtype=np.float64), cells, np.asarray(facet_list, dtype=np.int64),
                      cell_facets, facet_cells, interior_index, interior_facets,
                      np.asarray(ekeys, dtype=np.int64), cell_edges, colour)


def edge_patches(topo: Topology3D, dpf: int) -> List:
    """Ordered list of (edge, dof index array) for the non-empty edge patches: the patch of
    edge e holds every unknown on the interior faces containing e (Section 3.4.2 with the
    edge in place of the vertex).  Order: by colour, then edge id; faces in increasing
    interior number inside a patch."""
    inc = [[] for _ in range(topo.edges.shape[0])]
    eid = {tuple(e): i for i, e in enumerate(topo.edges.tolist())}
    for i, F in enumerate(topo.interior_facets):
        a, b, c = (int(v) for v in topo.facets[F])
        for e in ((a, b), (a, c), (b, c)):
            inc[eid[e]].append(i)
    order = sorted(range(len(inc)), key=lambda e: (int(topo.edge_colour[e]), e))
    out = []
    for e in order:
        if inc[e]:
            fac = sorted(inc[e])
            dofs = np.concatenate([np.arange(f * dpf, (f + 1) * dpf) for f in fac])
            out.append((e, dofs))
    return out
