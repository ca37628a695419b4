"""Host-side 3D topology of the library (no GPU): hdg_check_hierarchy on tetrahedral
hierarchies builds faces, edge patches with their greedy colouring and the transfer slots of
Bey's red refinement, and its sizes agree with the oracle's topology; malformed hierarchies
are rejected with a reason."""
import numpy as np
import pytest

from workloads.mesh3d import unit_cube_hierarchy
from oracle.topology3d import build_topology_3d, edge_patches


def _hdg():
    hdg = pytest.importorskip("paper_2303_06762_gb300")
    try:
        hdg.load_library()
    except Exception as e:          # library not built in this environment
        pytest.skip(f"library not available: {e}")
    return hdg


@pytest.mark.parametrize("n0,nl,kw", [(1, 3, {}), (2, 2, dict(jitter=0.2, seed=2, shuffle_seed=3)), (3, 2, {})])
def test_check_hierarchy_matches_oracle_topology(n0, nl, kw):
    hdg = _hdg()
    ms = unit_cube_hierarchy(n0, nl, **kw)
    for k in (0, 2, 3):
        info = hdg.hdg_check_hierarchy(ms, k)
        t = build_topology_3d(ms[-1].coords, ms[-1].cells)
        pts = edge_patches(t, 3)
        assert info["n_interior_facets"] == t.n_interior
        assert info["n_dof"] == t.n_interior * 3 * (k + 1) * (k + 2) // 2
        assert info["n_patches"] == len(pts)
        assert info["n_colours"] == int(t.edge_colour.max()) + 1
        assert info["max_patch_facets"] == max(len(d) for _, d in pts) // 3
        assert info["max_patch_cells"] == 6


def test_rejects_non_red_refinement():
    hdg = _hdg()
    ms = unit_cube_hierarchy(1, 2)
    ms[1].parent = np.zeros(ms[1].n_cells, dtype=np.int32)     # every fine cell in coarse cell 0
    with pytest.raises(hdg.HdgError) as e:
        hdg.hdg_check_hierarchy(ms, 1)
    assert "eight children" in str(e.value)
