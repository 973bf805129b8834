"""The C-ABI library loads and exports every entry point declared in include/*.h (no GPU
needed: no compute call is made)."""
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(bi_\w+)\s*\(", src, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_functions()
    for n in ("bi_setup", "bi_matvec", "bi_solve", "bi_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2210_04892_gb300 import build
    lib = build.build()
    import ctypes
    L = ctypes.CDLL(lib)
    for n in declared_functions():
        assert hasattr(L, n), n


def test_binding_lists_every_symbol():
    from paper_2210_04892_gb300 import bi
    assert sorted(bi.EXPORTS) == declared_functions()


def test_setup_rejects_bad_arguments_without_gpu_work():
    """Argument validation happens before any device call."""
    import ctypes
    import numpy as np
    from paper_2210_04892_gb300 import bi
    L = bi.load()
    p = bi.default_params()
    assert p.digits == 3 and abs(p.leaf_box - 0.25) < 1e-15 and p.interp_order == 10
    h = ctypes.c_void_p()
    v = np.zeros((3, 3))
    t = np.zeros((1, 3), np.int32)
    assert L.bi_setup(v.ctypes.data, 3, t.ctypes.data, 1, 1.0, 3, ctypes.byref(p), ctypes.byref(h)) == bi.BI_ERR_ARG
    p.interp_order = 1
    v4 = np.zeros((4, 3))
    t4 = np.zeros((4, 3), np.int32)
    assert L.bi_setup(v4.ctypes.data, 4, t4.ctypes.data, 4, 1.0, 3, ctypes.byref(p), ctypes.byref(h)) == bi.BI_ERR_ARG
    assert b"out of range" in L.bi_last_error(None)
    assert L.bi_matvec(None, None, None, 1) == bi.BI_ERR_ARG
