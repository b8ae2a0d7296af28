"""Matrix-free finite-element operators on hybrid tetrahedral grids for GB300 (sm_103a).

Python face of the C library in ``csrc/`` (interface: ``include/hhg.h``).  The
classes below only marshal torch tensors (device memory, streams) into the C
calls; every step of the computation runs in the library's CUDA kernels.

    mesh = Mesh(vertices, tets, level)                 # Section 2: macro mesh refined to `level`
    op = Operator(mesh, degree=2, coeff=("sin3",), quad_degree=4)
    y = op.apply(x)                                    # y = A(k) x  (Eq. 4.1)
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import (HHG_F32, HHG_F64, HHG_DIFFUSION, HHG_EPSILON, HHG_DIRICHLET, HHG_NEUMANN, HHG_COEFF_CONST,
                   HHG_COEFF_SIN3, HHG_COEFF_FIELD_P1, HHG_COEFF_FIELD_P2, HHGError, check, lib)

__all__ = ["Mesh", "Operator", "CurlCurl", "HHGError", "lib", "dtype_code"]


def dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float64:
        return HHG_F64
    if t.dtype == torch.float32:
        return HHG_F32
    raise TypeError("tensors must be float32 or float64, got %s" % t.dtype)


def _dev_ptr(t: torch.Tensor) -> int:
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _stream(device=None) -> int:
    return torch.cuda.current_stream(device).cuda_stream


class Mesh:
    """A macro mesh refined uniformly to ``level`` (all levels 0..level available)."""

    def __init__(self, vertices, tets, level: int):
        v = np.ascontiguousarray(vertices, dtype=np.float64)
        t = np.ascontiguousarray(tets, dtype=np.int32)
        h = ctypes.c_void_p()
        check(lib.hhg_mesh_create(v.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(v),
                                  t.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), len(t), int(level),
                                  ctypes.byref(h)), "hhg_mesh_create")
        self.handle = h
        self.level = int(level)
        self.nmacro = len(t)
        self.device = torch.device("cuda", torch.cuda.current_device())

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            lib.hhg_mesh_destroy(h)
            self.handle = None

    def vec_size(self, degree: int, level: int | None = None) -> int:
        n = ctypes.c_int64()
        check(lib.hhg_vec_size(self.handle, self.level if level is None else level, degree, ctypes.byref(n)),
              "hhg_vec_size")
        return n.value

    def dof_count(self, degree: int, level: int | None = None):
        tot, inn = ctypes.c_int64(), ctypes.c_int64()
        check(lib.hhg_dof_count(self.handle, self.level if level is None else level, degree, ctypes.byref(tot),
                                ctypes.byref(inn)), "hhg_dof_count")
        return tot.value, inn.value

    def empty(self, degree: int, dtype=torch.float64, level: int | None = None, per_point: int = 1):
        return torch.empty(self.vec_size(degree, level) * per_point, dtype=dtype, device=self.device)

    def coordinates(self, degree: int, level: int | None = None) -> torch.Tensor:
        """Physical coordinates (npoints, 3) of the packed points of a degree-p space."""
        lvl = self.level if level is None else level
        xyz = torch.empty(self.vec_size(degree, lvl) * 3, dtype=torch.float64, device=self.device)
        check(lib.hhg_vec_coordinates(self.handle, lvl, degree, _dev_ptr(xyz), _stream()), "hhg_vec_coordinates")
        return xyz.view(-1, 3)

    def make_consistent(self, x: torch.Tensor, degree: int, level: int | None = None, per_point: int = 1):
        check(lib.hhg_vec_make_consistent(self.handle, self.level if level is None else level, degree, _dev_ptr(x),
                                          dtype_code(x), per_point, _stream()), "hhg_vec_make_consistent")
        return x

    def dot(self, x: torch.Tensor, y: torch.Tensor, degree: int, level: int | None = None, per_point: int = 1):
        r = ctypes.c_double()
        check(lib.hhg_vec_dot(self.handle, self.level if level is None else level, degree, _dev_ptr(x), _dev_ptr(y),
                              dtype_code(x), per_point, ctypes.byref(r), _stream()), "hhg_vec_dot")
        return r.value

    def prolongate(self, xc: torch.Tensor, degree: int, level_fine: int, out: torch.Tensor | None = None):
        out = self.empty(degree, xc.dtype, level_fine) if out is None else out
        check(lib.hhg_prolongate(self.handle, level_fine, degree, _dev_ptr(xc), _dev_ptr(out), dtype_code(xc),
                                 _stream()), "hhg_prolongate")
        return out

    def restrict(self, rf: torch.Tensor, degree: int, level_fine: int, out: torch.Tensor | None = None):
        out = self.empty(degree, rf.dtype, level_fine - 1) if out is None else out
        check(lib.hhg_restrict(self.handle, level_fine, degree, _dev_ptr(rf), _dev_ptr(out), dtype_code(rf),
                               _stream()), "hhg_restrict")
        return out

    def prolongate_edges(self, xc: torch.Tensor, level_fine: int, out: torch.Tensor | None = None):
        out = self.empty(2, xc.dtype, level_fine) if out is None else out
        check(lib.hhg_prolongate_edges(self.handle, level_fine, _dev_ptr(xc), _dev_ptr(out), dtype_code(xc),
                                       _stream()), "hhg_prolongate_edges")
        return out

    def restrict_edges(self, rf: torch.Tensor, level_fine: int, out: torch.Tensor | None = None):
        out = self.empty(2, rf.dtype, level_fine - 1) if out is None else out
        check(lib.hhg_restrict_edges(self.handle, level_fine, _dev_ptr(rf), _dev_ptr(out), dtype_code(rf), _stream()),
              "hhg_restrict_edges")
        return out

    def gradient(self, p: torch.Tensor, level: int | None = None, out: torch.Tensor | None = None):
        lvl = self.level if level is None else level
        out = self.empty(2, p.dtype, lvl) if out is None else out
        check(lib.hhg_gradient(self.handle, lvl, _dev_ptr(p), _dev_ptr(out), dtype_code(p), _stream()), "hhg_gradient")
        return out

    def gradient_transpose(self, e: torch.Tensor, level: int | None = None, out: torch.Tensor | None = None):
        lvl = self.level if level is None else level
        out = self.empty(1, e.dtype, lvl) if out is None else out
        check(lib.hhg_gradient_transpose(self.handle, lvl, _dev_ptr(e), _dev_ptr(out), dtype_code(e), _stream()),
              "hhg_gradient_transpose")
        return out

    def rhs_sin3_poisson(self, degree: int, level: int | None = None):
        lvl = self.level if level is None else level
        b = self.empty(degree, torch.float64, lvl)
        check(lib.hhg_rhs_sin3_poisson(self.handle, lvl, degree, _dev_ptr(b), _stream()), "hhg_rhs_sin3_poisson")
        return b

    def l2_error_sin3(self, uh: torch.Tensor, degree: int, level: int | None = None) -> float:
        r = ctypes.c_double()
        check(lib.hhg_l2_error_sin3(self.handle, self.level if level is None else level, degree, _dev_ptr(uh),
                                    ctypes.byref(r), _stream()), "hhg_l2_error_sin3")
        return r.value


_COEFF_TYPES = {"const": HHG_COEFF_CONST, "sin3": HHG_COEFF_SIN3, "field_p1": HHG_COEFF_FIELD_P1,
                "field_p2": HHG_COEFF_FIELD_P2}


class Operator:
    """A matrix-free operator y = A(k) x on a mesh (Eq. 4.1).

    coeff: ("const", value) | ("sin3",) | ("field_p1", tensor) | ("field_p2", tensor); a field
    tensor is borrowed (kept referenced here) and read at every apply.
    """

    def __init__(self, mesh: Mesh, kind: str = "diffusion", degree: int = 1, coeff=("const", 1.0),
                 bc: str = "dirichlet", quad_degree: int = 2, level: int | None = None):
        self.mesh = mesh
        self.kind = {"diffusion": HHG_DIFFUSION, "epsilon": HHG_EPSILON}[kind]
        self.degree = degree
        self.level = mesh.level if level is None else level
        self.ncomp = 3 if kind == "epsilon" else 1
        c = _lib.hhg_coeff_t()
        c.type = _COEFF_TYPES[coeff[0]]
        self.field = None
        if coeff[0] == "const":
            c.value = float(coeff[1])
        elif coeff[0].startswith("field"):
            self.field = coeff[1]
            c.field = _dev_ptr(self.field)
            c.field_dtype = dtype_code(self.field)
        self.coeff = coeff
        h = ctypes.c_void_p()
        check(lib.hhg_op_create(mesh.handle, self.level, self.kind, degree, ctypes.byref(c),
                                {"dirichlet": HHG_DIRICHLET, "neumann": HHG_NEUMANN}[bc], quad_degree,
                                ctypes.byref(h)), "hhg_op_create")
        self.handle = h
        self.bc = bc

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            lib.hhg_op_destroy(h)
            self.handle = None

    def set_fp64_arith(self, mode: str) -> "Operator":
        """"native" (FP64 operations, the default) or "double_float" (FP64 vectors, FP32-pair
        arithmetic; P1 and P2 constant-coefficient diffusion)."""
        code = {"native": 0, "double_float": 1}[mode]
        check(lib.hhg_op_set_fp64_arith(self.handle, code), "hhg_op_set_fp64_arith")
        return self

    def set_field(self, field: torch.Tensor):
        self.field = field
        check(lib.hhg_op_set_field(self.handle, _dev_ptr(field), dtype_code(field)), "hhg_op_set_field")

    def vec_size(self) -> int:
        return self.mesh.vec_size(self.degree, self.level) * self.ncomp

    def apply(self, x: torch.Tensor, out: torch.Tensor | None = None, nrhs: int = 1) -> torch.Tensor:
        out = torch.empty_like(x) if out is None else out
        check(lib.hhg_op_apply(self.handle, _dev_ptr(x), _dev_ptr(out), dtype_code(x), nrhs, _stream()),
              "hhg_op_apply")
        return out

    def adjoint_coeff(self, u: torch.Tensor, g: torch.Tensor, out: torch.Tensor | None = None,
                      nrhs: int = 1) -> torch.Tensor:
        if out is None:
            out = torch.empty_like(self.field) if self.field is not None else torch.empty_like(u)
        check(lib.hhg_op_apply_adjoint_coeff(self.handle, _dev_ptr(u), _dev_ptr(g), _dev_ptr(out), dtype_code(u),
                                             nrhs, _stream()), "hhg_op_apply_adjoint_coeff")
        return out

    def store_element_matrices(self, dtype=torch.float64) -> "Operator":
        """Precomputed variant: integrate the local matrices once; applies in ``dtype`` read them."""
        check(lib.hhg_op_store_element_matrices(self.handle, HHG_F64 if dtype == torch.float64 else HHG_F32,
                                                _stream()), "hhg_op_store_element_matrices")
        return self

    def drop_element_matrices(self) -> "Operator":
        check(lib.hhg_op_drop_element_matrices(self.handle), "hhg_op_drop_element_matrices")
        return self

    def diagonal(self, dtype=torch.float64) -> torch.Tensor:
        d = self.mesh.empty(self.degree, dtype, self.level)
        check(lib.hhg_op_diagonal(self.handle, _dev_ptr(d), dtype_code(d), _stream()), "hhg_op_diagonal")
        return d

    def cheb_smooth(self, b, x, dinv, lam, lo=0.1, hi=1.1, order=2):
        check(lib.hhg_cheb_smooth(self.handle, _dev_ptr(b), _dev_ptr(x), _dev_ptr(dinv), float(lam), float(lo),
                                  float(hi), int(order), dtype_code(x), _stream()), "hhg_cheb_smooth")
        return x

    def power_iteration(self, dinv, v, iters: int) -> float:
        lam = ctypes.c_double()
        check(lib.hhg_power_iteration(self.handle, _dev_ptr(dinv), _dev_ptr(v), int(iters), dtype_code(v),
                                      ctypes.byref(lam), _stream()), "hhg_power_iteration")
        return lam.value

    def mg_solve(self, b: torch.Tensor, x: torch.Tensor, **opts):
        o = _lib.hhg_mg_opts_t()
        check(lib.hhg_mg_default_opts(ctypes.byref(o)), "hhg_mg_default_opts")
        for k, v in opts.items():
            setattr(o, k, v)
        st = _lib.hhg_mg_stats_t()
        code = lib.hhg_mg_solve(self.handle, _dev_ptr(b), _dev_ptr(x), ctypes.byref(o), ctypes.byref(st), _stream())
        stats = {"iterations": st.iterations, "rel_residual": st.rel_residual,
                 "history": list(st.residual_history[:max(1, min(64, st.iterations + 1))]),
                 "setup_ms": st.setup_ms, "solve_ms": st.solve_ms, "status": code}
        check(code, "hhg_mg_solve")
        return x, stats


class CurlCurl(Operator):
    """Lowest-order Nedelec operator alpha curl curl + beta (Eq. N1) on the micro-edges.

    Vectors use the degree-2 packed layout (edge-midpoint entries; vertex entries zero).
    alpha, beta: ("const", value) or ("field_p1", tensor) -- a P1 packed vector, borrowed.
    """

    def __init__(self, mesh: Mesh, alpha=("const", 1.0), beta=("const", 1.0), bc: str = "dirichlet",
                 level: int | None = None):
        self.mesh = mesh
        self.kind = _lib.HHG_CURLCURL
        self.degree = 2
        self.level = mesh.level if level is None else level
        self.ncomp = 1
        self.field = None
        self.fields = []
        cs = []
        for spec in (alpha, beta):
            c = _lib.hhg_coeff_t()
            c.type = _COEFF_TYPES[spec[0]]
            if spec[0] == "const":
                c.value = float(spec[1])
            else:
                self.fields.append(spec[1])
                c.field = _dev_ptr(spec[1])
                c.field_dtype = dtype_code(spec[1])
            cs.append(c)
        h = ctypes.c_void_p()
        check(lib.hhg_op_create_curlcurl(mesh.handle, self.level, ctypes.byref(cs[0]), ctypes.byref(cs[1]),
                                         {"dirichlet": HHG_DIRICHLET, "neumann": HHG_NEUMANN}[bc], ctypes.byref(h)),
              "hhg_op_create_curlcurl")
        self.handle = h
        self.bc = bc
        self.coeff = (alpha, beta)
