"""The C-ABI library loads and exports every function include/*.h declares (no GPU needed)."""
import ctypes
import glob
import os
import re

import pytest

import paper_1606_07550_gb300 as gpr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                             text, flags=re.M):
            if m.group(1) not in ("if", "while", "for", "return", "sizeof"):
                names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def built_lib():
    if not os.path.exists(gpr.LIB_PATH):
        gpr.build()
    return ctypes.CDLL(gpr.LIB_PATH)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("graph_build", "graph_free", "graph_info", "graph_export", "pagerank", "gpr_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(built_lib):
    missing = [n for n in declared_functions() if not hasattr(built_lib, n)]
    assert not missing, missing


def test_binding_loads_and_reports_errors_without_gpu_work():
    L = gpr.lib()
    assert isinstance(L.gpr_last_error(), bytes)  # (an earlier test on this thread may have left a message)
    # argument validation happens on the host, before any device call
    h = ctypes.c_void_p()
    assert L.graph_build(None, None, 5, 0, 0, None, ctypes.byref(h)) == gpr.EINVAL
    assert b"n = 0" in L.gpr_last_error()
    assert L.graph_build(None, None, 5, 10, 0, None, ctypes.byref(h)) == gpr.EINVAL
    assert L.pagerank(None, 0.85, 10, 0, 0, None, None, None) == gpr.EINVAL
    # the newer entry points check their arguments on the host as well
    assert L.ppr_target(None, 0, 0.85, 1e-4, None, 1, 10, 1, None, None, 0, None) == gpr.EINVAL
    assert L.ppr_reverse_push(None, 0, 0.85, 1e-4, None, None, None, 0, None) == gpr.EINVAL
    assert L.hits(None, 5, None, None, 0, None) == gpr.EINVAL
    assert L.eigen_centrality(None, 5, None, 0, None) == gpr.EINVAL
    assert L.wcc(None, None, None, 0, None) == gpr.EINVAL
    assert L.graph_update(None, None, None, 0, None, None, 0, 0, None) == gpr.EINVAL
    assert L.graph_save(None, b"/nonexistent/x") == gpr.EINVAL


def test_binding_checks_types_before_the_library():
    import numpy as np

    class NoGraph:  # any use of the handle would fail loudly
        @property
        def handle(self):
            raise AssertionError("the library was reached")

    g = NoGraph()
    with pytest.raises(ValueError):  # sources must be int32, estimates float64
        gpr.ppr_target(g, 0, np.zeros(3, np.int64), np.zeros(3), 1e-4, 10)
    with pytest.raises(ValueError):
        gpr.ppr_target(g, 0, np.zeros(3, np.int32), np.zeros(3, np.float32), 1e-4, 10)
    with pytest.raises(ValueError):  # lengths differ
        gpr.ppr_target(g, 0, np.zeros(3, np.int32), np.zeros(4), 1e-4, 10)
    with pytest.raises(ValueError):
        gpr.ppr_reverse_push(g, 0, 1e-4, np.zeros(3, np.float32))
    with pytest.raises(ValueError):  # an unknown schedule
        gpr.hits(g, np.zeros(3, np.float32), np.zeros(3, np.float32), spmv="sideways")
    with pytest.raises(ValueError):
        gpr.pagerank(g, np.zeros(3, np.float32), spmv="sideways")
    # the known names map to the header's flags
    from paper_1606_07550_gb300 import SPMV_BLOCKED, SPMV_PULL, _spmv_flag
    assert (_spmv_flag("auto"), _spmv_flag("pull"), _spmv_flag("blocked")) == (0, SPMV_PULL, SPMV_BLOCKED)
