"""The C-ABI library loads and exports every entry point declared in include/*.h (no GPU
needed: no compute call is made)."""
import glob
import os
import re


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


def test_every_entry_point_rejects_null_handles():
    """The error contract of the header: a NULL handle, server or plan (or a NULL output)
    gives BI_ERR_ARG, never a crash; the void entry points accept NULL.  No device call is
    made, so this runs without a GPU."""
    from paper_2210_04892_gb300 import bi
    L = bi.load()
    E = bi.BI_ERR_ARG
    assert L.bi_num_unknowns(None, None, None) == E
    assert L.bi_rwg_edges(None, None) == E
    assert L.bi_get_info(None, None) == E
    assert L.bi_matvec(None, None, None, 1) == E
    assert L.bi_matvec_host(None, None, None, 1) == E
    assert L.bi_rhs_planewave(None, None, None, 1, None) == E
    assert L.bi_solve(None, None, None, 1, 1e-3, None, None) == E
    assert L.bi_solve_refined(None, None, None, None, 1, 1e-3, None, None) == E
    assert L.bi_coupling_blocks(None, 0, None, None, None, None, None, None, None) == E
    assert L.bi_server_stats(None, None, 0) == E
    assert L.bi_set_coupling(None, 1, None, None, None, None, None, None, bi.QSOLVE(), None) == E
    assert L.bi_matvec_coupled(None, None, None, 1) == E
    assert L.bi_farfield(None, None, 1, None, 1, None) == E
    assert L.bi_farfield_noalloc(None, None, 1, None, 1, None) == E
    assert L.bi_debug_copy(None, 0, 0, None, 0) == E
    assert L.bi_debug_set_wait_limit(None, 1) == E
    assert L.bi_tuned_config(None, None, 0) == E
    assert L.bi_profile_stages(None, None, None, 1, 1, None) == E
    assert L.bi_device_status(None) == E
    L.bi_destroy(None)
    assert L.bi_server_create(None, None) == E
    assert L.bi_submit(None, None, 0, None, 0, 1.0, None, 1, None, None, 1e-3, None) == E
    assert L.bi_poll(None, 0, None, None) == E
    assert L.bi_result(None, 0, None, 0, None, None, None, None) == E
    assert L.bi_release(None, 0) == E
    assert L.bi_server_last_error(None) == b""
    L.bi_server_destroy(None)
    assert L.bi_plan_info(None, None) == E
    assert L.bi_plan_get(None, 0, 0, None, 0, None) == E
    L.bi_plan_destroy(None)
    assert L.bi_stage_name(0) == b"gather" and L.bi_stage_name(-1) == b"" and L.bi_stage_name(8) == b""
