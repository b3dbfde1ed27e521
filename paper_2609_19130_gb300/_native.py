"""ctypes view of libibf.so (include/ibf.h).  Argument marshalling only.

The library is built in-tree by paper_2609_19130_gb300.build; importing this
module loads it and raises if it is missing: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libibf.so")

IBF_OK = 0
IBF_ERR_INVALID_ARG = 1
IBF_ERR_UNSUPPORTED_SIZE = 2
IBF_ERR_OOM = 3
IBF_ERR_CUDA = 4
IBF_ERR_TIMEOUT = 5
IBF_ERR_NONFINITE = 6
IBF_WARN_INCOMPATIBLE_RHS = 7
IBF_ERR_UNSUPPORTED_BC = 8

IBF_BC_PERIODIC, IBF_BC_NEUMANN, IBF_BC_DIRICHLET = 0, 1, 2
IBF_FP64, IBF_MIXED = 0, 1
IBF_P_PHI, IBF_P_EXPLICIT, IBF_P_IMPLICIT = 0, 1, 2
IBF_MAX_GRIDS = 4096

# every entry point declared in include/ibf.h
EXPORTS = ("ibf_projection_plan", "ibf_project", "ibf_project_backward", "ibf_plan_sync_status",
           "ibf_plan_destroy", "ibf_status_string", "ibf_last_error", "ibf_plan_get_info",
           "ibf_profile_enable", "ibf_profile_read", "ibf_profile_reset", "ibf_project_noalloc",
           "ibf_projection_plan_tuned", "ibf_plan_get_tuning", "ibf_viscous_solve")


class ibf_grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("lx", C.c_double), ("ly", C.c_double), ("lz", C.c_double),
                ("zf", C.POINTER(C.c_double)), ("beta", C.c_double),
                ("bc_x", C.c_int), ("bc_y", C.c_int), ("bc_zlo", C.c_int), ("bc_zhi", C.c_int)]


class ibf_opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("refine_steps", C.c_int), ("autotune", C.c_int), ("pressure", C.c_int),
                ("inv_re", C.c_double)]


class ibf_fields(C.Structure):
    _fields_ = [("u", C.c_void_p), ("v", C.c_void_p), ("w", C.c_void_p), ("p", C.c_void_p), ("q", C.c_void_p)]


class ibf_stats(C.Structure):
    _fields_ = [("max_div", C.c_void_p), ("max_div_in", C.c_void_p), ("compat", C.c_void_p)]


class ibf_plan_info(C.Structure):
    _fields_ = [("workspace_bytes", C.c_longlong), ("ngrids", C.c_int), ("precision", C.c_int),
                ("refine_steps", C.c_int), ("total_cells", C.c_longlong)]


class ibf_tuning(C.Structure):
    _fields_ = [("rows", C.c_int), ("x_n1", C.c_int), ("y_n1", C.c_int), ("yz_kernel", C.c_int),
                ("mb", C.c_int), ("tri", C.c_int)]


TUNING_FIELDS = tuple(f for f, _ in ibf_tuning._fields_)


class IBFError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        msg = status_string(status)
        extra = last_error()
        super().__init__(f"{what}: {msg}" + (f" ({extra})" if extra else ""))


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libibf.so not built ({LIB_PATH}); run __graft_entry__.build() "
                              "or python -m paper_2609_19130_gb300.build")
        L = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        L.ibf_projection_plan.argtypes = [C.POINTER(vp), C.POINTER(ibf_grid), C.c_int, C.POINTER(ibf_opts), C.c_int]
        L.ibf_projection_plan.restype = C.c_int
        L.ibf_project.argtypes = [vp, C.POINTER(ibf_fields), C.POINTER(ibf_fields), C.c_double, C.c_double,
                                  C.POINTER(ibf_stats), vp]
        L.ibf_project.restype = C.c_int
        L.ibf_project_backward.argtypes = [vp, C.POINTER(ibf_fields), C.POINTER(ibf_fields), C.c_double,
                                           C.c_double, vp]
        L.ibf_project_backward.restype = C.c_int
        L.ibf_viscous_solve.argtypes = [vp, C.POINTER(ibf_fields), C.POINTER(ibf_fields), C.c_double, vp]
        L.ibf_viscous_solve.restype = C.c_int
        L.ibf_plan_sync_status.argtypes = [vp]
        L.ibf_plan_sync_status.restype = C.c_int
        L.ibf_plan_destroy.argtypes = [vp]
        L.ibf_plan_destroy.restype = C.c_int
        L.ibf_status_string.argtypes = [C.c_int]
        L.ibf_status_string.restype = C.c_char_p
        L.ibf_last_error.argtypes = []
        L.ibf_last_error.restype = C.c_char_p
        L.ibf_plan_get_info.argtypes = [vp, C.POINTER(ibf_plan_info)]
        L.ibf_plan_get_info.restype = C.c_int
        L.ibf_profile_enable.argtypes = [vp, C.c_int]
        L.ibf_profile_enable.restype = C.c_int
        L.ibf_profile_read.argtypes = [vp, C.POINTER(C.c_char_p), C.POINTER(C.c_longlong),
                                       C.POINTER(C.c_double), C.c_int]
        L.ibf_profile_read.restype = C.c_int
        L.ibf_profile_reset.argtypes = [vp]
        L.ibf_profile_reset.restype = C.c_int
        L.ibf_project_noalloc.argtypes = [C.POINTER(ibf_grid), C.POINTER(ibf_opts), C.POINTER(ibf_fields),
                                          C.POINTER(ibf_fields), C.c_double, C.c_double, vp]
        L.ibf_project_noalloc.restype = C.c_int
        L.ibf_projection_plan_tuned.argtypes = [C.POINTER(vp), C.POINTER(ibf_grid), C.c_int, C.POINTER(ibf_opts),
                                                C.c_int, C.POINTER(ibf_tuning)]
        L.ibf_projection_plan_tuned.restype = C.c_int
        L.ibf_plan_get_tuning.argtypes = [vp, C.c_int, C.POINTER(ibf_tuning)]
        L.ibf_plan_get_tuning.restype = C.c_int
        _lib = L
    return _lib


def status_string(s: int) -> str:
    return lib().ibf_status_string(int(s)).decode()


def last_error() -> str:
    return lib().ibf_last_error().decode()


def check(status: int, what: str = "ibf"):
    if status != IBF_OK:
        raise IBFError(status, what)
