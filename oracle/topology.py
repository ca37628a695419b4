"""Mesh topology for triangulations (oracle; test infrastructure only).

Conventions (they fix the layout of every skeleton vector):

* A facet (edge) is identified by its sorted global vertex pair; facets are
  numbered in lexicographic order of that pair.
* Local facet f of a cell is the facet opposite local vertex f.
* A facet is oriented from its lower to its higher global vertex id: unit
  tangent t_F = (x_hi - x_lo)/|F|, unit normal n_F = (t_y, -t_x); the facet
  parameter s ∈ [0,1] runs from x_lo to x_hi.
* Boundary facets (one adjacent cell) carry the homogeneous Dirichlet
  condition (Section 3.1) and hold no unknowns; interior facets are numbered
  in increasing facet id and own the skeleton unknowns.
"""

from __future__ import annotations

from dataclasses import dataclass
from typing import List

import numpy as np


@dataclass
class Topology:
    coords: np.ndarray          # (nv, 2)
    cells: np.ndarray           # (nc, 3)
    facets: np.ndarray          # (nf, 2) sorted vertex pairs
    cell_facets: np.ndarray     # (nc, 3) facet id opposite local vertex f
    facet_cells: np.ndarray     # (nf, 2) adjacent cells (second = -1 on the boundary)
    interior_index: np.ndarray  # (nf,) interior number or -1
    interior_facets: np.ndarray  # (n_int,) facet ids of interior facets
    vertex_colour: np.ndarray   # (nv,) proper vertex colouring

    @property
    def n_cells(self) -> int:
        return int(self.cells.shape[0])

    @property
    def n_interior(self) -> int:
        return int(self.interior_facets.shape[0])

    def facet_geometry(self, F: int):
        """(x_lo, x_hi, length, t_F, n_F) of facet F."""
        lo, hi = self.facets[F]
        xl, xh = self.coords[lo], self.coords[hi]
        d = xh - xl
        L = float(np.hypot(d[0], d[1]))
        t = d / L
        n = np.array([t[1], -t[0]])
        return xl, xh, L, t, n

    def cell_area(self, c: int) -> float:
        X = self.coords[self.cells[c]]
        J = np.stack([X[1] - X[0], X[2] - X[0]], axis=1)
        return 0.5 * abs(np.linalg.det(J))


def greedy_vertex_colouring(nv: int, edges: np.ndarray) -> np.ndarray:
    """Smallest-available-colour greedy colouring, vertices in increasing id."""
    adj: List[List[int]] = [[] for _ in range(nv)]
    for a, b in edges:
        adj[int(a)].append(int(b))
        adj[int(b)].append(int(a))
    colour = -np.ones(nv, dtype=np.int32)
    for v in range(nv):
        used = {int(colour[w]) for w in adj[v] if colour[w] >= 0}
        c = 0
        while c in used:
            c += 1
        colour[v] = c
    return colour


def build_topology(coords: np.ndarray, cells: np.ndarray, vertex_colour=None) -> Topology:
    cells = np.asarray(cells, dtype=np.int64)
    nc = cells.shape[0]
    keys = {}
    for c in range(nc):
        for f in range(3):
            a, b = [int(cells[c, i]) for i in range(3) if i != f]
            keys.setdefault((min(a, b), max(a, b)), []).append((c, f))
    facet_list = sorted(keys.keys())
    fid = {key: i for i, key in enumerate(facet_list)}
    nf = len(facet_list)
    cell_facets = np.empty((nc, 3), dtype=np.int64)
    facet_cells = -np.ones((nf, 2), dtype=np.int64)
    for key, lst in keys.items():
        F = fid[key]
        cs = sorted(c for c, _ in lst)
        if len(cs) > 2:
            raise ValueError("non-manifold facet")
        facet_cells[F, :len(cs)] = cs
        for c, f in lst:
            cell_facets[c, f] = F
    interior = facet_cells[:, 1] >= 0
    interior_facets = np.nonzero(interior)[0]
    interior_index = -np.ones(nf, dtype=np.int64)
    interior_index[interior_facets] = np.arange(interior_facets.shape[0])
    facets = np.asarray(facet_list, dtype=np.int64)
    if vertex_colour is None:
        vertex_colour = greedy_vertex_colouring(coords.shape[0], facets)
    return Topology(np.asarray(coords, dtype=np.float64), cells, facets, cell_facets,
                    facet_cells, interior_index, interior_facets,
                    np.asarray(vertex_colour, dtype=np.int32))
