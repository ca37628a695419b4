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
