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
    mat = vec = scales = 0
    for v in range(t.coords.shape[0]):
        if nf[v] == 0:
            continue
        npv = nf[v] * dpf
        mat += nf[v] * 2 * dpf * nloc + npv * npv      # two cells' rows per facet, the patch inverse
        vec += nc[v] * nloc + 3 * npv                  # gathered star unknowns, rhs, update
        scales += nf[v] * 2 * dpf + npv                # one scale per 16-bit row read
    assert bench.sweep_bytes(mesh, k, 4) == 4 * (mat + vec)
    assert bench.sweep_bytes(mesh, k, 8) == 8 * (mat + vec)
    assert bench.sweep_bytes(mesh, k, 4, 2) == 2 * mat + 4 * vec + 4 * scales


@pytest.mark.parametrize("N,k", [(4, 1), (8, 3), (6, 2)])
def test_full_size_counts_match_the_mesh(N, k):
    """The reference arm reports the GPU arm's config, whose skeleton size it computes
    in closed form: check the formula against the mesh."""
    t = topo_of(unit_square(N))
    assert bench.full_skeleton_dofs(N, k) == len(t.interior_facets) * 2 * (k + 1)
