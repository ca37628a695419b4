"""Structured triangulations of the unit square and their red-refinement hierarchy.

The meshes are the synthetic stand-ins for the paper's mesh sequences
T_1 ⊂ ... ⊂ T_J (Section 3.4.2), refined by joining edge midpoints
(Section 5.1.1).  A mesh is plain data: vertex coordinates, cell→vertex
connectivity, the parent cell of every cell on the next coarser level, and an
optional proper vertex colouring.  Nothing here knows about finite elements.

Two generators are provided:

* ``unit_square(N)``: N×N squares, each split by its (1,1) diagonal into two
  triangles (2N² cells).  Vertex (i, j) has id j·(N+1)+i; square (i, j) yields
  cells 2(jN+i) = (v(i,j), v(i+1,j), v(i+1,j+1)) and 2(jN+i)+1 =
  (v(i,j), v(i+1,j+1), v(i,j+1)).  The colouring (i+j) mod 3 is proper for the
  vertex graph of this triangulation.
* ``red_refine(mesh)``: splits every triangle into four through its edge
  midpoints, for arbitrary (e.g. jittered) coarse meshes.

The uniform refinement of ``unit_square(N)`` is, as a point set and cell set,
``unit_square(2N)``; ``unit_square_hierarchy`` uses the direct structured
numbering on every level and supplies the parent map by index arithmetic.
"""

from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np


@dataclass
class Mesh2D:
    coords: np.ndarray                 # (n_vertices, 2) float64
    cells: np.ndarray                  # (n_cells, 3) int32, local vertex order
    parent: Optional[np.ndarray] = None        # (n_cells,) int32 cell of the coarser level
    vertex_colour: Optional[np.ndarray] = None  # (n_vertices,) int32 proper colouring or None
    N: Optional[int] = None            # squares per side for structured meshes
    meta: dict = field(default_factory=dict)

    @property
    def n_vertices(self) -> int:
        return int(self.coords.shape[0])

    @property
    def n_cells(self) -> int:
        return int(self.cells.shape[0])


def unit_square(N: int, shuffle_seed: Optional[int] = None) -> Mesh2D:
    """Structured N×N triangulation of [0,1]² (2N² cells).

    ``shuffle_seed`` permutes the local vertex order of every cell with a
    seeded RNG; this changes orientations, not the triangulation.
    """
    if N < 1:
        raise ValueError("N must be >= 1")
    i, j = np.meshgrid(np.arange(N + 1), np.arange(N + 1), indexing="xy")
    coords = np.stack([i.ravel() / N, j.ravel() / N], axis=1).astype(np.float64)

    def vid(ii, jj):
        return jj * (N + 1) + ii

    si, sj = np.meshgrid(np.arange(N), np.arange(N), indexing="xy")
    si = si.ravel()
    sj = sj.ravel()
    lower = np.stack([vid(si, sj), vid(si + 1, sj), vid(si + 1, sj + 1)], axis=1)
    upper = np.stack([vid(si, sj), vid(si + 1, sj + 1), vid(si, sj + 1)], axis=1)
    cells = np.empty((2 * N * N, 3), dtype=np.int32)
    cells[0::2] = lower
    cells[1::2] = upper
    if shuffle_seed is not None:
        rng = np.random.default_rng(shuffle_seed)
        for c in range(cells.shape[0]):
            cells[c] = cells[c][rng.permutation(3)]
    colour = ((i.ravel() + j.ravel()) % 3).astype(np.int32)
    return Mesh2D(coords=coords, cells=cells, vertex_colour=colour, N=N)


def _structured_parent(N_fine: int) -> np.ndarray:
    """Parent map of unit_square(N_fine) into unit_square(N_fine // 2)."""
    Nc = N_fine // 2
    si, sj = np.meshgrid(np.arange(N_fine), np.arange(N_fine), indexing="xy")
    si = si.ravel()
    sj = sj.ravel()
    csq = (sj // 2) * Nc + (si // 2)
    di = si % 2
    dj = sj % 2
    parent = np.empty(2 * N_fine * N_fine, dtype=np.int32)
    # lower-right fine triangle (type 0) / upper-left (type 1) inside the
    # sub-square (di, dj) of the coarse square split by its (1,1) diagonal.
    t0 = np.where((di == 0) & (dj == 1), 1, 0)
    t1 = np.where((di == 1) & (dj == 0), 0, 1)
    parent[0::2] = 2 * csq + t0
    parent[1::2] = 2 * csq + t1
    return parent


def red_refine(mesh: Mesh2D) -> Mesh2D:
    """Split every triangle into four through its edge midpoints.

    For coarse cell (a, b, c) with midpoints m_ab, m_bc, m_ca the children
    are, in this order, (a, m_ab, m_ca), (m_ab, b, m_bc), (m_ca, m_bc, c) and
    (m_ab, m_bc, m_ca); they keep the orientation of the parent.
    """
    cells = mesh.cells
    nv = mesh.n_vertices
    edge_id = {}
    mids = []
    fine = []
    for c in range(cells.shape[0]):
        row = []
        for a, b in ((0, 1), (1, 2), (2, 0)):
            va, vb = int(cells[c, a]), int(cells[c, b])
            key = (min(va, vb), max(va, vb))
            if key not in edge_id:
                edge_id[key] = nv + len(mids)
                mids.append(0.5 * (mesh.coords[va] + mesh.coords[vb]))
            row.append(edge_id[key])
        a, b, cc = (int(v) for v in cells[c])
        mab, mbc, mca = row
        fine.extend([(a, mab, mca), (mab, b, mbc), (mca, mbc, cc), (mab, mbc, mca)])
    coords = np.vstack([mesh.coords, np.asarray(mids)]) if mids else mesh.coords.copy()
    fine_cells = np.asarray(fine, dtype=np.int32)
    parent = np.repeat(np.arange(cells.shape[0], dtype=np.int32), 4)
    return Mesh2D(coords=coords, cells=fine_cells, parent=parent)


def unit_square_hierarchy(N0: int, n_levels: int, shuffle_seed: Optional[int] = None,
                          jitter: float = 0.0, seed: int = 0) -> List[Mesh2D]:
    """Meshes T_1 (N0×N0) ... T_J (N0·2^(J-1)) with parent maps.

    With ``jitter`` > 0 the interior vertices of T_1 are moved by a seeded
    uniform perturbation of at most ``jitter``/N0 per coordinate and the finer
    levels are red refinements (no structured numbering, no colouring).
    """
    if jitter == 0.0:
        levels = []
        for l in range(n_levels):
            N = N0 * (2 ** l)
            m = unit_square(N, shuffle_seed=None if shuffle_seed is None else shuffle_seed + l)
            if l > 0:
                m.parent = _structured_parent(N)
            levels.append(m)
        return levels
    base = unit_square(N0)
    rng = np.random.default_rng(seed)
    x = base.coords.copy()
    interior = (x[:, 0] > 0) & (x[:, 0] < 1) & (x[:, 1] > 0) & (x[:, 1] < 1)
    x[interior] += rng.uniform(-jitter / N0, jitter / N0, size=(int(interior.sum()), 2))
    levels = [Mesh2D(coords=x, cells=base.cells.copy())]
    for _ in range(1, n_levels):
        levels.append(red_refine(levels[-1]))
    if shuffle_seed is not None:
        rng2 = np.random.default_rng(shuffle_seed)
        for m in levels:
            for c in range(m.n_cells):
                m.cells[c] = m.cells[c][rng2.permutation(3)]
    return levels


def step_channel(h: float = 0.5, length: float = 4.0, step_length: float = 1.0,
                 step_height: float = 0.5) -> Mesh2D:
    """Backward-facing-step channel (0, length) x (0, 1) without the step block
    (0, step_length) x (0, step_height): squares of side h (the step corners on the grid),
    each split by its (1,1) diagonal like ``unit_square``; vertices numbered row by row
    after removing the unused ones.  The colouring (i+j) mod 3 of the grid indices stays
    proper on the subset."""
    nx, ny = int(round(length / h)), int(round(1.0 / h))
    sx, sy = int(round(step_length / h)), int(round(step_height / h))
    keep_sq = np.ones((ny, nx), dtype=bool)
    keep_sq[:sy, :sx] = False
    used = np.zeros((ny + 1, nx + 1), dtype=bool)
    cells = []
    for j in range(ny):
        for i in range(nx):
            if not keep_sq[j, i]:
                continue
            used[j:j + 2, i:i + 2] = True
            cells.append(((i, j), (i + 1, j), (i + 1, j + 1)))
            cells.append(((i, j), (i + 1, j + 1), (i, j + 1)))
    ids = -np.ones((ny + 1, nx + 1), dtype=np.int64)
    jj, ii = np.nonzero(used)
    ids[jj, ii] = np.arange(len(jj))
    coords = np.stack([ii * h, jj * h], axis=1).astype(np.float64)
    cell_arr = np.array([[ids[b, a] for (a, b) in c] for c in cells], dtype=np.int32)
    colour = ((ii + jj) % 3).astype(np.int32)
    return Mesh2D(coords=coords, cells=cell_arr, vertex_colour=colour, meta={"h": h})


def step_channel_hierarchy(n_levels: int, h0: float = 0.5) -> List[Mesh2D]:
    """Levels of the backward-facing-step channel: ``step_channel(h0)`` refined by
    ``red_refine`` (greedy colouring on the finer levels)."""
    levels = [step_channel(h0)]
    for _ in range(1, n_levels):
        levels.append(red_refine(levels[-1]))
    return levels


def disjoint_union(hierarchies: List[List[Mesh2D]], gap: float = 0.5) -> List[Mesh2D]:
    """One hierarchy holding several meshes side by side, level by level: mesh i is shifted by
    i·(1 + gap) in x, its vertex and cell ids follow those of meshes 0..i-1, parent maps and
    vertex colourings are concatenated.  Every hierarchy needs the same number of levels.
    Because each mesh's vertex ids precede the next mesh's, the lexicographic facet numbering
    keeps every mesh's facets (and so its skeleton unknowns) in one contiguous block, in mesh
    order; cells likewise."""
    nl = len(hierarchies[0])
    if any(len(h) != nl for h in hierarchies):
        raise ValueError("all hierarchies need the same number of levels")
    out = []
    for l in range(nl):
        coords, cells, parent, colour = [], [], [], []
        voff = coff = pcoff = 0
        for i, h in enumerate(hierarchies):
            m = h[l]
            coords.append(m.coords + np.array([i * (1.0 + gap), 0.0]))
            cells.append(m.cells.astype(np.int64) + voff)
            if l > 0:
                parent.append(m.parent.astype(np.int64) + pcoff)
                pcoff += h[l - 1].n_cells
            col = m.vertex_colour if m.vertex_colour is not None else None
            colour.append(col)
            voff += m.n_vertices
            coff += m.n_cells
        vc = None if any(c is None for c in colour) else np.concatenate(colour).astype(np.int32)
        out.append(Mesh2D(coords=np.vstack(coords), cells=np.vstack(cells).astype(np.int32),
                          parent=np.concatenate(parent).astype(np.int32) if l > 0 else None,
                          vertex_colour=vc, meta={"parts": [h[l].n_cells for h in hierarchies]}))
    return out


def interior_facet_count(cells: np.ndarray) -> int:
    """Interior facets of a triangulation: (3 n_cells - n_boundary) / 2."""
    e = np.sort(np.concatenate([cells[:, [1, 2]], cells[:, [0, 2]], cells[:, [0, 1]]]).astype(np.int64), axis=1)
    _, cnt = np.unique(e, axis=0, return_counts=True)
    return int((cnt == 2).sum())
