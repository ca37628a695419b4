"""The algorithmic bytes behind the roofline of bench.py, recounted patch by patch from
the oracle's topology (vertex patches, their interior facets and star cells)."""
import numpy as np
import pytest

import bench
from workloads import unit_square
from _util import topo_of


@pytest.mark.parametrize("N,k,shuffle", [(4, 3, None), (6, 2, 3), (5, 1, 7)])
def test_sweep_bytes_counts_every_patch(N, k, shuffle):
    mesh = unit_square(N, shuffle_seed=shuffle) if shuffle else unit_square(N)
    t = topo_of(mesh)
    dpf, nloc = 2 * (k + 1), 6 * (k + 1)
    nf = np.zeros(t.coords.shape[0], dtype=int)
    for F in t.interior_facets:
        for v in t.facets[F]:
            nf[v] += 1
    nc = np.bincount(np.asarray(t.cells).ravel(), minlength=t.coords.shape[0])
    mat = vec = scales = closed = 0
    for v in range(t.coords.shape[0]):
        if nf[v] == 0:
            continue
        npv = nf[v] * dpf
        mat += nf[v] * 2 * dpf * nloc + npv * npv      # two cells' rows per facet, the patch inverse
        vec += nc[v] * nloc + 3 * npv                  # gathered star unknowns, rhs, update
        scales += nf[v] * 2 * dpf + npv                # one scale per 16-bit row read
        # closed form: one dpf x dpf coupling block per (facet, cell), the packed inverse, the
        # unknowns on each star cell's facet opposite v, rhs read and update written
        closed += nf[v] * 2 * dpf * dpf + npv * (npv + 1) // 2 + nc[v] * dpf + 2 * npv
    assert bench.sweep_bytes(mesh, k, 4) == 4 * (mat + vec)
    assert bench.sweep_bytes(mesh, k, 8) == 8 * (mat + vec)
    assert bench.sweep_bytes(mesh, k, 4, 2) == 2 * mat + 4 * vec + 4 * scales
    assert bench.sweep_bytes(mesh, k, 4, packed_inverse=True, closed_form=True) == 4 * closed
    # the AL split: Q's nc columns of np_max rows, one AL-free entry per slot, nc FP64 flux weights
    np_max = nf.max() * dpf
    split = sum(4 * (nc[v] * np_max + 2 * nf[v]) + 8 * nc[v] for v in range(t.coords.shape[0]) if nf[v] > 0)
    assert bench.sweep_bytes(mesh, k, 4, packed_inverse=True, closed_form=True, al_split=True) == 4 * closed + split


@pytest.mark.parametrize("N,k", [(4, 1), (8, 3), (6, 2)])
def test_full_size_counts_match_the_mesh(N, k):
    """The reference arm reports the GPU arm's config, whose skeleton size it computes
    in closed form: check the formula against the mesh."""
    t = topo_of(unit_square(N))
    assert bench.full_skeleton_dofs(N, k) == len(t.interior_facets) * 2 * (k + 1)


@pytest.mark.parametrize("n,k", [(2, 1), (3, 3)])
def test_tetra_sweep_bytes_counts_every_edge_patch(n, k):
    """Both byte models of the 3D edge-patch sweep (FP32, correction form), recounted from the
    oracle's edge patches and the cells around each edge."""
    from workloads.mesh3d import unit_cube
    from oracle.topology3d import build_topology_3d, edge_patches
    mesh = unit_cube(n, shuffle_seed=2)
    t = build_topology_3d(mesh.coords, mesh.cells)
    dpf = 3 * (k + 1) * (k + 2) // 2
    nloc = 4 * dpf
    edges = [tuple(e) for e in t.edges.tolist()]
    star = {e: 0 for e in edges}
    for c in np.asarray(mesh.cells):
        for a in range(4):
            for b in range(a + 1, 4):
                star[tuple(sorted((int(c[a]), int(c[b]))))] += 1
    kernel = packed = 0
    for e, dofs in edge_patches(t, dpf):
        npv = len(dofs)
        nfac = npv // dpf
        # transposed inverse; both cells' row blocks of every patch face; the star cells'
        # unknowns; g read, u read and written
        kernel += npv * npv + 2 * nfac * nloc * dpf + star[edges[e]] * nloc + 3 * npv
        packed += npv * (npv + 1) // 2
    N = len(t.interior_facets) * dpf
    model = packed + len(mesh.cells) * nloc * (nloc + 1) // 2 + 3 * N
    assert bench.tetra_sweep_bytes(np.asarray(mesh.cells), k) == (4 * model, 4 * kernel)
