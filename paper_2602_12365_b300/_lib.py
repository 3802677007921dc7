"""ctypes declarations of the C ABI in include/fem_b300.h.

Argument marshalling only: every step of the computation runs in the CUDA
library.  Importing this module loads ``libfem_b300.so`` and raises if it is
missing -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfem_b300.so")

FEM_OK = 0
STATUS_NAMES = {0: "FEM_OK", 1: "FEM_ERR_ARG", 2: "FEM_ERR_CUDA", 3: "FEM_ERR_INVERTED",
                4: "FEM_ERR_NONFINITE", 5: "FEM_ERR_NOT_CONVERGED", 6: "FEM_ERR_NEG_CURVATURE",
                7: "FEM_ERR_TIMEOUT", 8: "FEM_ERR_BADMESH", 9: "FEM_ERR_NOT_SPD",
                10: "FEM_ERR_LINESEARCH"}
FEM_F64, FEM_F32 = 0, 1
FEM_PREC_FP64, FEM_PREC_MIXED = 0, 1
FEM_MASK_OUT, FEM_MASK_IN = 1, 2
FEM_FLAG_INVERTED, FEM_FLAG_NONFINITE, FEM_FLAG_TIMEOUT = 1, 2, 4


class MeshDesc(C.Structure):
    _fields_ = [("elem_type", C.c_int32), ("precision", C.c_int32), ("n_nodes", C.c_int64),
                ("n_elems", C.c_int64), ("coords", C.c_void_p), ("conn", C.c_void_p),
                ("mu", C.c_void_p), ("lam", C.c_void_p), ("mu0", C.c_double),
                ("lambda0", C.c_double), ("dirichlet", C.c_void_p), ("tile_elems", C.c_int32),
                ("reserved", C.c_int32)]


class MeshInfo(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("n_elems", C.c_int64), ("dim", C.c_int32),
                ("n_en", C.c_int32), ("n_tiles", C.c_int32), ("max_tile_nodes", C.c_int32),
                ("n_rounds", C.c_int64), ("max_rounds", C.c_int32), ("n_shared", C.c_int32),
                ("n_slots", C.c_int64), ("n_local_nodes", C.c_int64), ("n_orphans", C.c_int64),
                ("round_fill", C.c_double), ("device_bytes", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


FEM_PC_BLOCK_JACOBI, FEM_PC_LEARNED = 0, 1
FEM_LP_FEATURES, FEM_LP_PARAMS = 36, 6918
FEM_LP_LOSS_RESIDUAL, FEM_LP_LOSS_ENERGY = 0, 1


class NewtonOpts(C.Structure):
    _fields_ = [("cg_dtype", C.c_int32), ("precond", C.c_int32), ("newton_rtol", C.c_double),
                ("newton_max", C.c_int32), ("ls_max", C.c_int32), ("eta_max", C.c_double),
                ("cg_max", C.c_int64), ("predictor_rtol", C.c_double), ("armijo_c", C.c_double),
                ("max_bisect", C.c_int32), ("cg_batch", C.c_int32), ("learned", C.c_void_p)]


class NewtonStats(C.Structure):
    _fields_ = [("status", C.c_int32), ("newton_iters", C.c_int32), ("cg_iters", C.c_int64),
                ("bisections", C.c_int32), ("ls_halvings", C.c_int32), ("r0_norm", C.c_double),
                ("r_norm", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class FemError(RuntimeError):
    def __init__(self, status, msg):
        self.status = status
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")


_lib = None


def lib():
    """The loaded library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing; build it with "
                              "`python -m paper_2602_12365_b300.build` (no CPU fallback exists)")
        L = C.CDLL(LIB_PATH)
        P, i32, u32 = C.c_void_p, C.c_int32, C.c_uint32
        L.fem_last_error.restype = C.c_char_p
        L.fem_last_error.argtypes = []
        sig = {
            "fem_mesh_create": [C.POINTER(MeshDesc), C.POINTER(C.c_void_p), P],
            "fem_mesh_destroy": [P],
            "fem_mesh_get_info": [P, C.POINTER(MeshInfo)],
            "fem_plan_partition": [C.POINTER(MeshDesc), P, P, P, P, C.POINTER(MeshInfo)],
            "fem_energy": [P, i32, P, P, P],
            "fem_energy_static": [P, i32, P, P, P],
            "fem_residual": [P, i32, P, P, u32, P],
            "fem_hvp": [P, i32, P, P, P, u32, P, P],
            "fem_block_diag": [P, i32, P, P, P],
            "fem_param_vjp": [P, i32, P, P, P, P, P],
            "fem_sync_status": [P, P, C.POINTER(i32)],
            "fem_newton_default_opts": [C.POINTER(NewtonOpts)],
            "fem_tangent_solve": [P, i32, P, P, P, C.c_double, C.c_int64, C.POINTER(C.c_int64), P],
            "fem_lp_create": [C.c_uint64, C.POINTER(C.c_void_p)],
            "fem_lp_destroy": [P],
            "fem_lp_set_loss": [P, i32],
            "fem_lp_set_clip": [P, C.c_float],
            "fem_lp_get_params": [P, P],
            "fem_lp_set_params": [P, P],
            "fem_lp_features": [P, P, P, P],
            "fem_lp_blocks": [P, P, P, P, P],
            "fem_lp_train_step": [P, P, P, P, C.c_float, C.POINTER(C.c_double), P],
            "fem_lp_gradient": [P, P, P, P, P, C.POINTER(C.c_double), P],
            "fem_newton_step": [P, P, P, C.c_double, C.c_double, C.POINTER(NewtonOpts),
                                C.POINTER(NewtonStats), P],
            "fem_sparse_info": [P, C.POINTER(C.c_int64), C.POINTER(i32)],
            "fem_sparse_pattern": [P, P, P, P],
            "fem_sparse_pattern_desc": [C.POINTER(MeshDesc), C.POINTER(C.c_int64), C.POINTER(i32), P, P, P],
            "fem_sparse_assemble": [P, i32, P, u32, P, P],
            "fem_sparse_spmv": [P, i32, P, P, P, P],
            "fem_residual_atomic": [P, i32, P, P, u32, P],
            "fem_mesh_set_ncm": [P, i32, P],
            "fem_hvp_atomic": [P, i32, P, P, P, u32, P],
            "fem_sparse_assemble_atomic": [P, i32, P, u32, P, P],
            "fem_compliance_gradient": [P, P, C.c_double, C.c_double, i32, i32, P, P, C.POINTER(C.c_int64), P],
            "fem_fp32_fma_rate": [i32, i32, P, C.POINTER(C.c_double), P],
            "fem_mesh_set_moduli": [P, P, P, P],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.restype = C.c_int
            fn.argtypes = args
        _lib = L
    return _lib


def check(status: int):
    if status != FEM_OK:
        raise FemError(status, lib().fem_last_error().decode())


# every symbol the header declares (checked by the CPU test suite)
EXPORTED = ["fem_mesh_create", "fem_mesh_destroy", "fem_mesh_get_info", "fem_plan_partition",
            "fem_energy", "fem_energy_static", "fem_residual", "fem_hvp", "fem_block_diag", "fem_param_vjp",
            "fem_sync_status", "fem_newton_default_opts", "fem_newton_step", "fem_tangent_solve",
            "fem_lp_create", "fem_lp_destroy", "fem_lp_set_loss", "fem_lp_set_clip",
            "fem_lp_get_params", "fem_lp_set_params",
            "fem_lp_features", "fem_lp_blocks", "fem_lp_gradient", "fem_lp_train_step",
            "fem_sparse_info", "fem_sparse_pattern", "fem_sparse_pattern_desc", "fem_sparse_assemble",
            "fem_sparse_spmv", "fem_residual_atomic", "fem_hvp_atomic", "fem_sparse_assemble_atomic",
            "fem_mesh_set_ncm", "fem_compliance_gradient", "fem_fp32_fma_rate", "fem_mesh_set_moduli",
            "fem_last_error"]
