"""Structured tetrahedrisations of the unit cube and their red-refinement hierarchy.

The 3D stand-ins for the paper's mesh sequences T_1 ⊂ ... ⊂ T_J (Section 3.4.2,
Section 5.1.2): plain data (vertex coordinates, cell→vertex connectivity, the parent
cell of every cell on the next coarser level).  Nothing here knows about finite elements.

* ``unit_cube(n)``: n³ cubes, each split into the 6 Kuhn tetrahedra that share the
  cube's main diagonal (6n³ cells).  Vertex (i, j, l) has id (l (n+1) + j)(n+1) + i.
  The tetrahedron of cube (i, j, l) for the axis permutation σ is the monotone path
  v, v + e_σ0, v + e_σ0 + e_σ1, v + (1, 1, 1) from the cube's lower corner v; the
  permutations are taken in lexicographic order.
* ``red_refine_3d(mesh)``: splits every tetrahedron (x0, x1, x2, x3) into eight
  through its edge midpoints x_ij: the four corner tetrahedra and the inner
  octahedron cut along the x02–x13 diagonal (Bey's rule), keeping the parent's
  vertex order in each child.  Applied to ``unit_cube(n)`` it yields the Kuhn
  tetrahedra of ``unit_cube(2n)`` (as sets of cells; the numbering differs).
"""

from __future__ import annotations

from dataclasses import dataclass, field
from itertools import permutations
from typing import List, Optional

import numpy as np


@dataclass
class Mesh3D:
    coords: np.ndarray                 # (n_vertices, 3) float64
    cells: np.ndarray                  # (n_cells, 4) int32, local vertex order
    parent: Optional[np.ndarray] = None        # (n_cells,) int32 cell of the coarser level
    n: Optional[int] = None            # cubes per side for the structured coarse mesh
    meta: dict = field(default_factory=dict)

    @property
    def n_vertices(self) -> int:
        return int(self.coords.shape[0])

    @property
    def n_cells(self) -> int:
        return int(self.cells.shape[0])

    # the 2D meshes' field; 3D hierarchies colour their edge patches instead
    vertex_colour = None


def unit_cube(n: int, shuffle_seed: Optional[int] = None) -> Mesh3D:
    """Kuhn tetrahedrisation of [0,1]³ with n cubes per side (6n³ cells).

    ``shuffle_seed`` permutes the local vertex order of every cell with a seeded
    RNG; this changes orientations, not the tetrahedrisation.
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    g = np.arange(n + 1)
    I, J, L = np.meshgrid(g, g, g, indexing="ij")
    coords = np.stack([I.ravel(order="F"), J.ravel(order="F"), L.ravel(order="F")], axis=1) / n

    def vid(i, j, l):
        return (l * (n + 1) + j) * (n + 1) + i

    ci, cj, cl = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ci, cj, cl = ci.ravel(order="F"), cj.ravel(order="F"), cl.ravel(order="F")
    cells = np.empty((6 * n ** 3, 4), dtype=np.int32)
    for t, perm in enumerate(permutations(range(3))):
        p = np.zeros(3, dtype=np.int64)
        cols = [vid(ci, cj, cl)]
        for ax in perm:
            p[ax] += 1
            cols.append(vid(ci + p[0], cj + p[1], cl + p[2]))
        cells[t::6] = np.stack(cols, axis=1)
    if shuffle_seed is not None:
        rng = np.random.default_rng(shuffle_seed)
        for c in range(cells.shape[0]):
            cells[c] = cells[c][rng.permutation(4)]
    return Mesh3D(coords=coords.astype(np.float64), cells=cells, n=n)


# Bey's children in terms of (vertex or midpoint) slots: 0..3 vertices, then the
# midpoints 01, 02, 03, 12, 13, 23 as slots 4..9
_EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))
_CHILDREN = ((0, 4, 5, 6), (4, 1, 7, 8), (5, 7, 2, 9), (6, 8, 9, 3),
             (4, 5, 6, 8), (4, 5, 7, 8), (5, 6, 8, 9), (5, 7, 8, 9))


def red_refine_3d(mesh: Mesh3D) -> Mesh3D:
    """Split every tetrahedron into eight through its edge midpoints (Bey's rule).

    Midpoint vertices are numbered after the coarse vertices, in lexicographic
    order of their sorted edge; the children of cell c are cells 8c .. 8c+7.
    """
    cells = mesh.cells.astype(np.int64)
    nc = cells.shape[0]
    e = np.stack([np.sort(cells[:, [a, b]], axis=1) for a, b in _EDGES], axis=1)   # (nc, 6, 2)
    uniq, inv = np.unique(e.reshape(-1, 2), axis=0, return_inverse=True)
    mid_id = mesh.n_vertices + inv.reshape(nc, 6)
    mids = 0.5 * (mesh.coords[uniq[:, 0]] + mesh.coords[uniq[:, 1]])
    slots = np.concatenate([cells, mid_id], axis=1)                                # (nc, 10)
    fine = slots[:, np.asarray(_CHILDREN)].reshape(-1, 4).astype(np.int32)
    coords = np.vstack([mesh.coords, mids])
    parent = np.repeat(np.arange(nc, dtype=np.int32), 8)
    return Mesh3D(coords=coords, cells=fine, parent=parent)


def unit_cube_hierarchy(n0: int, n_levels: int, jitter: float = 0.0, seed: int = 0,
                        shuffle_seed: Optional[int] = None) -> List[Mesh3D]:
    """Meshes T_1 (``unit_cube(n0)``) ... T_J (n0·2^(J-1) cubes per side) by red refinement.

    With ``jitter`` > 0 the interior vertices of T_1 are moved by a seeded uniform
    perturbation of at most ``jitter``/n0 per coordinate; ``shuffle_seed`` permutes
    the local vertex order of the cells of every level (seeded).
    """
    base = unit_cube(n0)
    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        x = base.coords
        interior = np.all((x > 0) & (x < 1), axis=1)
        x[interior] += rng.uniform(-jitter / n0, jitter / n0, size=(int(interior.sum()), 3))
    levels = [base]
    for _ in range(1, n_levels):
        levels.append(red_refine_3d(levels[-1]))
    if shuffle_seed is not None:
        rng2 = np.random.default_rng(shuffle_seed)
        for m in levels:
            for c in range(m.n_cells):
                m.cells[c] = m.cells[c][rng2.permutation(4)]
    return levels


def boundary_faces_3d(cells: np.ndarray) -> np.ndarray:
    """(n_boundary, 3) sorted global vertex triples of the boundary faces in face order
    (lexicographic in the sorted triple)."""
    f = np.concatenate([cells[:, [1, 2, 3]], cells[:, [0, 2, 3]], cells[:, [0, 1, 3]],
                        cells[:, [0, 1, 2]]]).astype(np.int64)
    f.sort(axis=1)
    uniq, cnt = np.unique(f, axis=0, return_counts=True)
    return uniq[cnt == 1]
