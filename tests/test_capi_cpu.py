"""The C library loads and exports every entry point of include/hhg.h; host-side argument checks (no GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import importlib.util
    spec = importlib.util.spec_from_file_location("_hhg_build", os.path.join(ROOT, "paper_2404_08371_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    path = mod.build()
    from paper_2404_08371_gb300 import _lib
    assert os.path.samefile(_lib.LIB, path)
    return _lib.lib


def declared_functions():
    text = open(os.path.join(ROOT, "include", "hhg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hhg_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    from paper_2404_08371_gb300 import _lib
    for n in names:
        assert hasattr(lib, n), n
        assert n in _lib.SIGNATURES, n


def _create(lib, v, t, level=2):
    from paper_2404_08371_gb300 import _lib
    v = np.ascontiguousarray(v, dtype=np.float64)
    t = np.ascontiguousarray(t, dtype=np.int32)
    h = ctypes.c_void_p()
    code = lib.hhg_mesh_create(v.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(v),
                               t.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), len(t), level, ctypes.byref(h))
    return code, h


def test_mesh_validation_errors(lib):
    from paper_2404_08371_gb300 import _lib
    ref = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]])
    # degenerate macro (coplanar vertices)
    code, _ = _create(lib, [[0, 0, 0], [1, 0, 0], [2, 0, 0], [0, 0, 1.0]], [[0, 1, 2, 3]])
    assert code == _lib.HHG_E_DEGENERATE and b"degenerate" in lib.hhg_last_error()
    # a face shared by three macros
    v = np.vstack([ref, [[0.3, 0.3, -1.0], [0.3, 0.3, -2.0]]])
    code, _ = _create(lib, v, [[0, 1, 2, 3], [0, 1, 2, 4], [0, 1, 2, 5]])
    assert code == _lib.HHG_E_NONMANIFOLD
    # index out of range, bad level
    code, _ = _create(lib, ref, [[0, 1, 2, 7]])
    assert code == _lib.HHG_E_ARG
    code, _ = _create(lib, ref, [[0, 1, 2, 3]], level=11)
    assert code == _lib.HHG_E_ARG


def test_null_arguments_rejected(lib):
    from paper_2404_08371_gb300 import _lib
    assert lib.hhg_op_apply(None, None, None, 1, 1, None) == _lib.HHG_E_ARG
    assert lib.hhg_vec_size(None, 0, 1, None) == _lib.HHG_E_ARG
    assert lib.hhg_mg_default_opts(None) == _lib.HHG_E_ARG
    assert lib.hhg_op_store_element_matrices(None, _lib.HHG_F64, None) == _lib.HHG_E_ARG
    assert lib.hhg_op_drop_element_matrices(None) == _lib.HHG_E_ARG
    o = _lib.hhg_mg_opts_t()
    assert lib.hhg_mg_default_opts(ctypes.byref(o)) == 0
    assert (o.nu1, o.nu2, o.cheb_order, o.power_iters, o.tol) == (2, 2, 2, 15, 1e-10)
