"""Host-side validation of hdg_setup_mesh_hierarchy: every check on the mesh hierarchy
(cell indices, facets, the proper vertex colouring that makes a colour phase of block
Gauss-Seidel race-free, the red-refinement parent maps) runs on the host before any
device call, so these run without a GPU."""
import copy

import numpy as np
import pytest

import paper_2303_06762_gb300 as hdg
from workloads import unit_square, unit_square_hierarchy


def _setup_error(levels):
    with pytest.raises(hdg.HdgError) as ei:
        hdg.hdg_setup_mesh_hierarchy(levels)
    assert ei.value.status == 1, str(ei.value)           # HDG_ERR_INVALID_ARG
    return str(ei.value)


def test_improper_colouring_is_rejected():
    m = copy.copy(unit_square(4))
    col = np.array(m.vertex_colour, dtype=np.int32)
    a, b = m.cells[0][:2]
    col[b] = col[a]                                       # two vertices of one cell share a colour
    m.vertex_colour = col
    assert "not proper" in _setup_error([m])


def test_colour_out_of_range_is_rejected():
    m = copy.copy(unit_square(3))
    col = np.array(m.vertex_colour, dtype=np.int32)
    col[0] = 300
    m.vertex_colour = col
    assert "colour out of range" in _setup_error([m])


def test_bad_cells_are_rejected():
    m = copy.copy(unit_square(3))
    cells = np.array(m.cells, dtype=np.int32)
    cells[2, 1] = m.coords.shape[0] + 5
    m.cells = cells
    assert "out of range" in _setup_error([m])
    m2 = copy.copy(unit_square(3))
    cells = np.array(m2.cells, dtype=np.int32)
    cells[1, 2] = cells[1, 0]
    m2.cells = cells
    assert "degenerate" in _setup_error([m2])


def test_non_nested_hierarchy_is_rejected():
    ms = [copy.copy(m) for m in unit_square_hierarchy(2, 3)]
    parent = np.array(ms[2].parent, dtype=np.int32)
    parent[0], parent[-1] = parent[-1], parent[0]         # two fine cells swap their coarse cells
    ms[2].parent = parent
    msg = _setup_error(ms)
    assert "level 2" in msg


@pytest.mark.parametrize("kw", [dict(), dict(shuffle_seed=4), dict(jitter=0.25, seed=3, shuffle_seed=5)])
@pytest.mark.parametrize("k", [0, 2])
def test_checked_hierarchy_sizes_match_the_oracle(kw, k):
    """hdg_check_hierarchy builds the library's host topology, patches and transfer tables
    without a GPU; its sizes agree with the oracle's topology and vertex patches."""
    from _util import hierarchy
    from oracle.mg import vertex_patches
    ms, ts, ps = hierarchy(2, 4, **kw)
    info = hdg.hdg_check_hierarchy(ms, k)
    t = ts[-1]
    patches = vertex_patches(t, 2 * (k + 1))
    assert info["n_levels"] == 4
    assert info["n_interior_facets"] == len(t.interior_facets)
    assert info["n_dof"] == len(t.interior_facets) * 2 * (k + 1)
    assert info["n_patches"] == len(patches)
    assert info["max_patch_facets"] == max(len(d) for _, d in patches) // (2 * (k + 1))
    cells_at = np.bincount(np.asarray(t.cells).ravel(), minlength=t.coords.shape[0])
    assert info["max_patch_cells"] == max(cells_at[v] for v, _ in patches)
    assert info["n_colours"] == len({int(t.vertex_colour[v]) for v, _ in patches})


def test_check_hierarchy_reports_the_reason():
    m = copy.copy(unit_square(4))
    col = np.array(m.vertex_colour, dtype=np.int32)
    a, b = m.cells[3][1:]
    col[b] = col[a]
    m.vertex_colour = col
    with pytest.raises(hdg.HdgError) as ei:
        hdg.hdg_check_hierarchy([m], 1)
    assert ei.value.status == 1 and "not proper" in str(ei.value)
