"""The C-ABI library builds, loads and exports every entry point declared in include/hdg.h
(no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1807_00086_gb300 import build, hdg
    if not os.path.exists(hdg.LIB_PATH):
        build.build()
    return hdg.LIB_PATH


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(hdg_\w+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("hdg_setup", "hdg_condense", "hdg_trace_solve", "hdg_recover", "hdg_step",
                     "hdg_trace_apply", "hdg_condensed_rhs"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(libpath):
    from paper_1807_00086_gb300 import hdg
    assert set(declared_functions()) <= set(hdg.SIGNATURES)
    hdg.load()


def test_default_options_without_gpu(libpath):
    from paper_1807_00086_gb300 import hdg
    lib = hdg.load()
    opt = hdg.Options()
    lib.hdg_default_options(ctypes.byref(opt))
    assert opt.prec == hdg.HDG_FP64 and opt.rtol == 1e-13 and opt.maxit > 0


def test_setup_rejects_bad_input_on_host(libpath):
    """Argument validation happens on the host before any device call."""
    import numpy as np
    from paper_1807_00086_gb300 import hdg
    lib = hdg.load()
    ctx = ctypes.c_void_p()
    vert = np.zeros((3, 2))
    elem = np.array([[0, 1, 2]], dtype=np.int32)
    rho = np.ones(1)
    mesh = hdg.Mesh(2, 3, 1, vert.ctypes.data_as(hdg.P_double), elem.ctypes.data_as(hdg.P_int32))
    mat = hdg.Material(0, rho.ctypes.data_as(hdg.P_double), rho.ctypes.data_as(hdg.P_double), None, None)
    st = lib.hdg_setup(ctypes.byref(mesh), 7, 1.0, ctypes.byref(mat), None, None, ctypes.byref(ctx))
    assert st == -1 and b"degree" in lib.hdg_last_error(ctx)
    lib.hdg_destroy(ctx)
    st = lib.hdg_setup(ctypes.byref(mesh), 2, 1.0, ctypes.byref(mat), None, None, ctypes.byref(ctx))
    assert st == -1 and b"degenerate" in lib.hdg_last_error(ctx)
    lib.hdg_destroy(ctx)


def test_setup_rejects_unsupported_elastic_configurations_on_host(libpath):
    import numpy as np
    from paper_1807_00086_gb300 import hdg, inputs
    lib = hdg.load()
    vert, elem = inputs.unit_cube_tet(1)
    ne = elem.shape[0]
    one = np.ones(ne)
    mesh = hdg.Mesh(3, vert.shape[0], ne, vert.ctypes.data_as(hdg.P_double), elem.ctypes.data_as(hdg.P_int32))
    mat = hdg.Material(1, one.ctypes.data_as(hdg.P_double), None, one.ctypes.data_as(hdg.P_double),
                       one.ctypes.data_as(hdg.P_double))
    ctx = ctypes.c_void_p()
    # per-element degrees: each in 1..4, 3D elastic only
    ks = np.full(ne, 2, dtype=np.int32)
    ks[3] = 5
    mesh.elem_k = ks.ctypes.data_as(hdg.P_int32)
    st = lib.hdg_setup(ctypes.byref(mesh), 4, 1.0, ctypes.byref(mat), None, None, ctypes.byref(ctx))
    assert st == -1 and b"1..4" in lib.hdg_last_error(ctx)
    lib.hdg_destroy(ctx)
    ks[3] = 1
    amat = hdg.Material(0, one.ctypes.data_as(hdg.P_double), one.ctypes.data_as(hdg.P_double), None, None)
    st = lib.hdg_setup(ctypes.byref(mesh), 2, 1.0, ctypes.byref(amat), None, None, ctypes.byref(ctx))
    assert st == -1 and b"3D elastic" in lib.hdg_last_error(ctx)
    lib.hdg_destroy(ctx)
    mesh.elem_k = None
    bad = -np.ones(ne)
    mat.mu = bad.ctypes.data_as(hdg.P_double)
    st = lib.hdg_setup(ctypes.byref(mesh), 2, 1.0, ctypes.byref(mat), None, None, ctypes.byref(ctx))
    assert st == -1 and b"Lame" in lib.hdg_last_error(ctx)
    lib.hdg_destroy(ctx)


def test_entry_points_reject_a_null_context_without_gpu(libpath):
    """Every context entry point returns HDG_EINVAL for a null context, before any CUDA call."""
    from paper_1807_00086_gb300 import hdg
    lib = hdg.load()
    names = ["hdg_get_sizes", "hdg_condense", "hdg_get_schur", "hdg_trace_apply", "hdg_condensed_rhs",
             "hdg_trace_solve", "hdg_recover", "hdg_postprocess", "hdg_set_sources", "hdg_quadrature_points",
             "hdg_project_volume", "hdg_set_dirichlet", "hdg_set_state", "hdg_get_state", "hdg_step",
             "hdg_reset_column", "hdg_get_tuning", "hdg_enable_stats", "hdg_get_stats"]
    for name in names:
        args = []
        for t in hdg.SIGNATURES[name][1]:
            if t in (ctypes.c_int32, ctypes.c_int64):
                args.append(0)
            elif t is ctypes.c_double:
                args.append(1.0)
            else:
                args.append(None)
        assert getattr(lib, name)(*args) == -1, name
    assert lib.hdg_last_error(None) == b"null context"
