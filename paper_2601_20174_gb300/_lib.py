"""ctypes binding of libnlsp.so (the C ABI declared in include/nlsp.h).

Argument marshalling only: every step of the solver runs in the CUDA library.
Loading fails loudly when the library has not been built; there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnlsp.so")

NLSP_OK = 0
NLSP_NOT_CONVERGED = 1
NLSP_ERR_INVALID = -1
NLSP_ERR_CUDA = -2
NLSP_ERR_NOT_SPD = -3
NLSP_ERR_BREAKDOWN = -4
NLSP_ERR_TIMEOUT = -5
NLSP_ERR_OOM = -6

NLSP_FP64 = 0
NLSP_MIXED_FP32 = 1
NLSP_MIXED_BF16 = 2
NLSP_MIXED_TF32 = 3

NLSP_COEF_CELL_KAPPA = 0
NLSP_COEF_CONST_TENSOR = 1


class SetupParams(C.Structure):
    _fields_ = [("K", C.c_int), ("k", C.c_int), ("s1", C.c_int), ("nu1", C.c_int), ("nu2", C.c_int),
                ("omega", C.c_double), ("precision", C.c_int), ("seed", C.c_ulonglong)]


NLSP_STREAM_S0 = 3


class SolveParams(C.Structure):
    _fields_ = [("tol", C.c_double), ("maxit", C.c_int), ("flexible", C.c_int), ("graph_mode", C.c_int)]


class SolveInfo(C.Structure):
    _fields_ = [("iterations", C.c_int), ("status", C.c_int), ("relres", C.c_double),
                ("true_relres", C.c_double)]


vp = C.c_void_p
i64 = C.c_int64
ci = C.c_int
cd = C.c_double

# name -> (restype, argtypes); mirrors include/nlsp.h
SIGNATURES = {
    "nlsp_status_string": (C.c_char_p, [ci]),
    "nlsp_last_error": (C.c_char_p, []),
    "nlsp_create": (ci, [C.POINTER(vp), ci, vp]),
    "nlsp_set_stream": (ci, [vp, vp]),
    "nlsp_destroy": (None, [vp]),
    "nlsp_assemble_stencil": (ci, [vp, ci, C.POINTER(i64), ci, vp, ci, C.POINTER(vp)]),
    "nlsp_assemble_csr": (ci, [vp, i64, i64, vp, vp, vp, C.POINTER(vp)]),
    "nlsp_op_size": (i64, [vp]),
    "nlsp_op_apply": (ci, [vp, vp, ci, vp, i64, vp, i64]),
    "nlsp_op_diagonal": (ci, [vp, vp, vp]),
    "nlsp_free_op": (None, [vp]),
    "nlsp_smooth_samples": (ci, [vp, vp, ci, ci, cd, ci, vp, vp]),
    "nlsp_build_prolongation": (ci, [vp, vp, C.POINTER(SetupParams), vp, C.POINTER(vp)]),
    "nlsp_build_prolongation_a_weighted": (ci, [vp, vp, C.POINTER(SetupParams), vp, C.POINTER(vp)]),
    "nlsp_build_prolongation_randomized": (ci, [vp, vp, C.POINTER(SetupParams), vp, ci, ci, vp, C.POINTER(vp)]),
    "nlsp_prec_from_basis": (ci, [vp, vp, C.POINTER(SetupParams), vp, ci, C.POINTER(vp)]),
    "nlsp_factor_coarse": (ci, [vp, vp, vp, ci]),
    "nlsp_prec_dims": (ci, [vp, C.POINTER(i64), C.POINTER(ci), C.POINTER(ci), C.POINTER(ci), C.POINTER(ci)]),
    "nlsp_prec_copy_basis": (ci, [vp, vp, vp]),
    "nlsp_prec_copy_sigma": (ci, [vp, vp, vp]),
    "nlsp_prec_copy_coarse": (ci, [vp, vp, vp, vp]),
    "nlsp_free_prec": (None, [vp]),
    "nlsp_apply_prec": (ci, [vp, vp, ci, vp, i64, vp, i64]),
    "nlsp_solve": (ci, [vp, vp, vp, ci, vp, i64, vp, i64, C.POINTER(SolveParams), C.POINTER(SolveInfo)]),
    "nlsp_launch_count": (C.c_ulonglong, [vp]),
    "nlsp_apply_prec_noalloc": (ci, [vp, vp, ci, vp, i64, vp, i64]),
    "nlsp_prec_phase_times": (ci, [vp, vp, C.POINTER(C.c_double), ci]),
    "nlsp_random_normal": (ci, [vp, C.c_ulonglong, C.c_ulonglong, C.c_ulonglong, i64, vp]),
    "nlsp_check_conversions": (ci, [vp, vp, i64, C.POINTER(C.c_ulonglong)]),
    "nlsp_bench_kernel": (ci, [vp, vp, ci, ci]),
    "nlsp_solve_batched": (ci, [vp, ci, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), C.POINTER(SolveParams), ci,
                                C.POINTER(SolveInfo)]),
    "nlsp_tune_batched": (ci, [vp, ci, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), C.POINTER(SolveParams),
                               C.POINTER(ci), ci, C.POINTER(ci), C.POINTER(cd)]),
    "nlsp_plan_teams": (ci, [ci, C.POINTER(i64), ci, ci, C.POINTER(ci), C.POINTER(ci), C.POINTER(cd)]),
    "nlsp_solve_block": (ci, [vp, vp, vp, ci, vp, i64, vp, i64, C.POINTER(SolveParams), C.POINTER(SolveInfo)]),
    "nlsp_solve_block_cg": (ci, [vp, vp, vp, ci, vp, i64, vp, i64, C.POINTER(SolveParams), C.POINTER(SolveInfo)]),
    "nlsp_subspace_loss": (ci, [vp, i64, ci, ci, ci, vp, vp, C.POINTER(cd), vp]),
    "nlsp_nlss_loss": (ci, [vp, i64, ci, ci, ci, vp, vp, C.POINTER(cd), vp]),
    "nlsp_unrolled_pcg": (ci, [vp, vp, vp, ci, ci, cd, ci, vp, ci, C.POINTER(cd), vp]),
}

_lib = None


class NlspError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = f"{where}: {status_string(status)}"
        last = last_error()
        if status == NLSP_ERR_CUDA and last:
            msg += f" ({last})"
        super().__init__(msg)


def load() -> C.CDLL:
    """Loads libnlsp.so; raises if it is missing (build it with
    paper_2601_20174_gb300.build.build() or __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: the CUDA library must be built "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def status_string(status: int) -> str:
    try:
        return load().nlsp_status_string(status).decode()
    except Exception:  # library not loadable: plain number
        return str(status)


def last_error() -> str:
    try:
        return load().nlsp_last_error().decode()
    except Exception:
        return ""


def check(status: int, where: str, allow=(NLSP_OK,)) -> int:
    if status not in allow:
        raise NlspError(status, where)
    return status
