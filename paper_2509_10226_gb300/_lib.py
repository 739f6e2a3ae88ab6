"""ctypes declarations of the tetmf C ABI (include/tetmf.h).

Argument marshalling only.  Loading fails loudly if the shared library has not
been built; there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import re

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libtetmf.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "tetmf.h")

FEM_OK, FEM_EINVAL, FEM_EMESH, FEM_EUNSUPPORTED, FEM_ECUDA, FEM_ENOTCONV, FEM_ENOMEM = range(7)
FEM_CG, FEM_DG = 0, 1
FEM_RULE_STANDARD, FEM_RULE_MODIFIED = 0, 1
FEM_SCATTER_ATOMIC, FEM_SCATTER_COLOUR = 0, 1
FEM_FP64, FEM_FP32, FEM_TF32, FEM_BF16, FEM_TF32X3 = 0, 1, 2, 3, 4
FEM_REORDER_NONE, FEM_REORDER_MORTON = 0, 1
FEM_SOLVE_FP64_PCG, FEM_SOLVE_IR_MIXED, FEM_SOLVE_IR_PMG = 0, 1, 2

STATUS_NAMES = {0: "FEM_OK", 1: "FEM_EINVAL", 2: "FEM_EMESH", 3: "FEM_EUNSUPPORTED", 4: "FEM_ECUDA",
                5: "FEM_ENOTCONV", 6: "FEM_ENOMEM"}


class FemError(RuntimeError):
    def __init__(self, status, func, message):
        super().__init__(f"{func}: {STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class MeshDesc(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_int64), ("xyz", ctypes.c_void_p), ("n_cells", ctypes.c_int64),
                ("cells", ctypes.c_void_p), ("cell_nodes", ctypes.c_void_p)]


class SpaceDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("degree", ctypes.c_int32), ("dirichlet", ctypes.c_int32),
                ("reorder", ctypes.c_int32), ("dg_penalty_factor", ctypes.c_double), ("device", ctypes.c_int32),
                ("cell_rule", ctypes.c_int32), ("scatter", ctypes.c_int32)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("inner_prec", ctypes.c_int32), ("rtol", ctypes.c_double),
                ("inner_rtol", ctypes.c_double), ("max_outer", ctypes.c_int32), ("max_inner", ctypes.c_int32),
                ("smoother_degree", ctypes.c_int32), ("coarse_steps", ctypes.c_int32)]


class SolveStats(ctypes.Structure):
    _fields_ = [("outer_iterations", ctypes.c_int32), ("inner_iterations", ctypes.c_int32),
                ("rel_residual", ctypes.c_double), ("seconds", ctypes.c_double)]


_P = ctypes.c_void_p
_SIGNATURES = {
    "fem_create": [ctypes.POINTER(MeshDesc), ctypes.POINTER(SpaceDesc), ctypes.POINTER(ctypes.c_void_p)],
    "fem_destroy": [_P],
    "fem_num_dofs": [_P, _P],
    "fem_num_cells": [_P, _P],
    "fem_dofs_per_cell": [_P, _P],
    "fem_num_qpoints": [_P, _P],
    "fem_num_faces": [_P, _P, _P],
    "fem_cell_permutation": [_P, _P],
    "fem_dof_permutation": [_P, _P],
    "fem_dof_keys": [_P, _P],
    "fem_dof_coordinates": [_P, _P],
    "fem_colours": [_P, _P, _P],
    "fem_transfer_create": [_P, _P, ctypes.POINTER(ctypes.c_void_p)],
    "fem_transfer_destroy": [_P],
    "fem_prolongate": [_P, ctypes.c_int32, _P, _P, _P],
    "fem_restrict": [_P, ctypes.c_int32, _P, _P, _P],
    "fem_apply_vector": [_P, ctypes.c_int32, ctypes.c_int32, _P, _P, _P],
    "fem_chebyshev": [_P, ctypes.c_int32, _P, _P, _P, ctypes.c_int32, ctypes.c_double, ctypes.c_double, _P, _P],
    "fem_lambda_max": [_P, ctypes.c_int32, _P, _P, ctypes.c_int32, _P, _P, _P],
    "fem_smoother_work_bytes": [_P, ctypes.c_int32, _P],
    "fem_dirichlet_mask": [_P, _P],
    "fem_device_status": [_P, _P],
    "fem_selftest_wait": [_P, ctypes.c_int64, _P],
    "fem_apply": [_P, ctypes.c_int32, _P, _P, _P, _P],
    "fem_apply_host": [_P, ctypes.c_int32, ctypes.c_int64, _P, _P],
    "fem_apply_adjoint": [_P, ctypes.c_int32, _P, _P, _P, _P],
    "fem_coeff_grad": [_P, ctypes.c_int32, _P, _P, _P, _P, _P, _P],
    "fem_diagonal": [_P, ctypes.c_int32, _P, _P, _P],
    "fem_rhs_const": [_P, ctypes.c_double, _P, _P],
    "fem_csr_build": [_P, _P],
    "fem_csr_apply": [_P, ctypes.c_int32, _P, _P, _P],
    "fem_solve": [_P, ctypes.POINTER(SolveOpts), _P, _P, ctypes.POINTER(SolveStats), _P],
    "fem_solve_noalloc": [_P, ctypes.POINTER(SolveOpts), _P, _P, ctypes.POINTER(SolveStats), _P],
    "fem_fma_probe": [ctypes.c_int32, ctypes.c_int64, _P, ctypes.POINTER(ctypes.c_double), _P],
}
FEM_SOLVE_NOALLOC_MAX_DOFS = 262144

_lib = None


def header_functions(path: str = HEADER):
    """Names of every function the public header declares."""
    with open(path) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\s*\*)\s*(fem_\w+)\s*\(", text, flags=re.M)))


def lib():
    """The loaded shared library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2509_10226_gb300.build` "
                              "(the CUDA library is required; there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.fem_last_error.argtypes = []
        L.fem_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def check(status: int, func: str):
    if status != FEM_OK:
        raise FemError(status, func, lib().fem_last_error().decode(errors="replace"))
    return status


def call(name: str, *args):
    return check(getattr(lib(), name)(*args), name)
