"""ctypes binding of the hhg C interface (include/hhg.h): argument marshalling only.

Every function of the header is exposed under its C name with its C
signature; the library is the in-tree build ``_build/libhhg.so``.  Importing
this module fails loudly when that library has not been built: there is no
other implementation to fall back to.
"""
from __future__ import annotations

import ctypes
import os

LIB = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "libhhg.so")

HHG_OK = 0
HHG_E_ARG, HHG_E_DEGENERATE, HHG_E_NONMANIFOLD, HHG_E_OOM, HHG_E_CUDA, HHG_E_NOT_CONVERGED, HHG_E_NAN, \
    HHG_E_UNSUPPORTED = -1, -2, -3, -4, -5, -6, -7, -8
HHG_F32, HHG_F64 = 0, 1
HHG_DIFFUSION, HHG_EPSILON, HHG_CURLCURL = 0, 1, 2
HHG_DIRICHLET, HHG_NEUMANN = 0, 1
HHG_COEFF_CONST, HHG_COEFF_SIN3, HHG_COEFF_FIELD_P1, HHG_COEFF_FIELD_P2 = 0, 1, 2, 3

_vp = ctypes.c_void_p
_i = ctypes.c_int
_i64 = ctypes.c_int64
_d = ctypes.c_double


class hhg_coeff_t(ctypes.Structure):
    _fields_ = [("type", _i), ("value", _d), ("field", _vp), ("field_dtype", _i)]


class hhg_mg_opts_t(ctypes.Structure):
    _fields_ = [("nu1", _i), ("nu2", _i), ("cheb_order", _i), ("power_iters", _i), ("cheb_lo", _d),
                ("cheb_hi", _d), ("tol", _d), ("max_iters", _i), ("mixed", _i), ("fmg", _i),
                ("coarse_level", _i)]


class hhg_mg_stats_t(ctypes.Structure):
    _fields_ = [("iterations", _i), ("rel_residual", _d), ("residual_history", _d * 64), ("setup_ms", _d),
                ("solve_ms", _d)]


SIGNATURES = {
    "hhg_last_error": ([], ctypes.c_char_p),
    "hhg_mesh_create": ([ctypes.POINTER(_d), _i64, ctypes.POINTER(ctypes.c_int32), _i64, _i, ctypes.POINTER(_vp)], _i),
    "hhg_mesh_destroy": ([_vp], _i),
    "hhg_vec_size": ([_vp, _i, _i, ctypes.POINTER(_i64)], _i),
    "hhg_dof_count": ([_vp, _i, _i, ctypes.POINTER(_i64), ctypes.POINTER(_i64)], _i),
    "hhg_op_create": ([_vp, _i, _i, _i, ctypes.POINTER(hhg_coeff_t), _i, _i, ctypes.POINTER(_vp)], _i),
    "hhg_op_create_curlcurl": ([_vp, _i, ctypes.POINTER(hhg_coeff_t), ctypes.POINTER(hhg_coeff_t), _i,
                                ctypes.POINTER(_vp)], _i),
    "hhg_op_destroy": ([_vp], _i),
    "hhg_op_set_field": ([_vp, _vp, _i], _i),
    "hhg_op_apply": ([_vp, _vp, _vp, _i, _i, _vp], _i),
    "hhg_op_apply_adjoint_coeff": ([_vp, _vp, _vp, _vp, _i, _i, _vp], _i),
    "hhg_op_diagonal": ([_vp, _vp, _i, _vp], _i),
    "hhg_op_store_element_matrices": ([_vp, _i, _vp], _i),
    "hhg_op_drop_element_matrices": ([_vp], _i),
    "hhg_vec_coordinates": ([_vp, _i, _i, _vp, _vp], _i),
    "hhg_vec_make_consistent": ([_vp, _i, _i, _vp, _i, _i, _vp], _i),
    "hhg_vec_dot": ([_vp, _i, _i, _vp, _vp, _i, _i, ctypes.POINTER(_d), _vp], _i),
    "hhg_prolongate": ([_vp, _i, _i, _vp, _vp, _i, _vp], _i),
    "hhg_restrict": ([_vp, _i, _i, _vp, _vp, _i, _vp], _i),
    "hhg_rhs_sin3_poisson": ([_vp, _i, _i, _vp, _vp], _i),
    "hhg_l2_error_sin3": ([_vp, _i, _i, _vp, ctypes.POINTER(_d), _vp], _i),
    "hhg_cheb_smooth": ([_vp, _vp, _vp, _vp, _d, _d, _d, _i, _i, _vp], _i),
    "hhg_cheb_smooth_noalloc": ([_vp, _vp, _vp, _vp, _d, _d, _d, _i, _i, _vp], _i),
    "hhg_power_iteration": ([_vp, _vp, _vp, _i, _i, ctypes.POINTER(_d), _vp], _i),
    "hhg_mg_default_opts": ([ctypes.POINTER(hhg_mg_opts_t)], _i),
    "hhg_mg_solve": ([_vp, _vp, _vp, ctypes.POINTER(hhg_mg_opts_t), ctypes.POINTER(hhg_mg_stats_t), _vp], _i),
    "hhg_op_set_fp64_arith": ([_vp, _i], _i),
    "hhg_prolongate_edges": ([_vp, _i, _vp, _vp, _i, _vp], _i),
    "hhg_restrict_edges": ([_vp, _i, _vp, _vp, _i, _vp], _i),
    "hhg_gradient": ([_vp, _i, _vp, _vp, _i, _vp], _i),
    "hhg_gradient_transpose": ([_vp, _i, _vp, _vp, _i, _vp], _i),
}


class HHGError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__("%s failed with status %d: %s" % (where, code, msg))
        self.code = code


def _load():
    if not os.path.exists(LIB):
        raise ImportError("libhhg.so is not built (%s); run `python -c \"import __graft_entry__ as g; g.build()\"` "
                          "or `python -m paper_2404_08371_gb300.build`" % LIB)
    lib = ctypes.CDLL(LIB)
    for name, (args, res) in SIGNATURES.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


lib = _load()


def check(code: int, where: str) -> None:
    if code != HHG_OK:
        raise HHGError(code, where, lib.hhg_last_error().decode())


def __getattr__(name):
    if name in SIGNATURES:
        return getattr(lib, name)
    raise AttributeError(name)
