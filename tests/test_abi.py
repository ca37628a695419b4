"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/hdg.h (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "hdg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hdg_[a-z0-9_]+)\s*\(", src)))


def test_build_and_exports():
    from paper_2303_06762_gb300.build import build
    path = build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    import paper_2303_06762_gb300 as hdg
    assert sorted(hdg.EXPORTS) == declared_functions()


def test_host_only_calls():
    """Calls that touch no device: status strings, default options, argument checks."""
    import paper_2303_06762_gb300 as hdg
    lib = hdg.load_library()
    assert lib.hdg_status_string(0) == b"ok"
    assert lib.hdg_status_string(4) == b"singular factorisation"
    o = hdg.SolveOpts()
    lib.hdg_default_solve_opts(ctypes.byref(o))
    assert (o.rtol, o.atol, o.restart) == (1e-8, 1e-10, 30)
    h = ctypes.c_void_p()
    assert lib.hdg_setup_mesh_hierarchy(None, 0, ctypes.byref(h)) == 1     # invalid argument
    assert lib.hdg_apply(None, None, None, None) == 1
