"""ctypes binding of libaao_rk.so: the C ABI of include/aao_rk.h, same names.

Argument marshalling only.  The library is loaded from this package
directory; if it is missing the import fails loudly (there is no fallback).
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libaao_rk.so")

AAO_OK = 0
STATUS = {0: "AAO_OK", -1: "AAO_ERR_ARG", -2: "AAO_ERR_CUDA", -3: "AAO_ERR_OOM",
          -4: "AAO_ERR_NOT_CONVERGED", -5: "AAO_ERR_BREAKDOWN", -6: "AAO_ERR_NONFINITE",
          -7: "AAO_ERR_TIMEOUT", -8: "AAO_ERR_UNSUPPORTED"}
PREC = {"fp64": 0, "fp32": 1, "bf16": 2, "fp16": 3}
DISC = {"fd": 0, "q1": 1}


class aao_grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("len", C.c_double * 3), ("disc", C.c_int),
                ("kappa", C.c_void_p)]


class aao_tableau(C.Structure):
    _fields_ = [("s", C.c_int), ("A", C.c_double * 64), ("b", C.c_double * 8), ("c", C.c_double * 8)]


class aao_options(C.Structure):
    _fields_ = [("tol", C.c_double), ("restart", C.c_int), ("maxit", C.c_int),
                ("inner_maxit", C.c_int), ("inner_tol", C.c_double),
                ("mg_cycles", C.c_int), ("mg_pre", C.c_int), ("mg_post", C.c_int),
                ("mg_omega", C.c_double), ("cheb_steps", C.c_int),
                ("prec_P", C.c_int), ("prec_Pint", C.c_int), ("ckpt_every", C.c_int),
                ("stream", C.c_void_p), ("mgrit_m", C.c_int), ("precond_side", C.c_int),
                ("relax_matvec", C.c_double)]


class aao_info(C.Structure):
    _fields_ = [("outer_its", C.c_int), ("inner_its_total", C.c_longlong), ("rel_res", C.c_double),
                ("converged", C.c_int), ("t_theta_ms", C.c_double), ("t_schur_ms", C.c_double),
                ("t_total_ms", C.c_double), ("n_history", C.c_int), ("history", C.c_double * 128),
                ("relaxed_matvecs", C.c_int)]


H = C.c_void_p
P = C.c_void_p   # double* (host or device address)

# (name, restype, argtypes) of every entry point declared in include/aao_rk.h
SIGNATURES = [
    ("aao_rk_default_options", None, [C.POINTER(aao_options)]),
    ("aao_rk_setup", C.c_int, [C.POINTER(aao_grid), C.c_double, C.c_int, C.POINTER(aao_tableau),
                               C.POINTER(aao_options), C.POINTER(H)]),
    ("aao_rk_destroy", None, [H]),
    ("aao_rk_last_error", C.c_char_p, []),
    ("aao_rk_launch_count", C.c_longlong, []),
    ("aao_rk_profile_begin", C.c_int, [C.c_char_p]),
    ("aao_rk_profile_end", C.c_int, [C.POINTER(C.c_longlong), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("aao_rk_profile_report", C.c_char_p, []),
    ("aao_rk_sizes", C.c_int, [H, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
    ("aao_rk_set_options", C.c_int, [H, C.POINTER(aao_options)]),
    ("aao_rk_rhs", C.c_int, [H, P, C.c_int, P, P]),
    ("aao_rk_matvec", C.c_int, [H, P, P]),
    ("aao_rk_matvec_transpose", C.c_int, [H, P, P]),
    ("aao_rk_matvec_relaxed", C.c_int, [H, P, P, P, C.c_int]),
    ("aao_rk_precond_apply", C.c_int, [H, P, P]),
    ("aao_rk_precond_apply_transpose", C.c_int, [H, P, P]),
    ("aao_rk_solve", C.c_int, [H, P, C.c_int, P, P, C.c_int, C.POINTER(aao_info)]),
    ("aao_rk_solve_rhs", C.c_int, [H, P, P, C.c_int, C.POINTER(aao_info)]),
    ("aao_rk_adjoint_solve", C.c_int, [H, P, P, P, P, P, C.POINTER(aao_info)]),
    ("aao_rk_grad_kappa", C.c_int, [H, P, P, P, C.c_int]),
    ("aao_rk_solve_batched", C.c_int, [C.c_int, C.POINTER(H), C.POINTER(P), C.POINTER(P), C.POINTER(P),
                                       C.POINTER(aao_info)]),
    ("aao_rk_shifted_solve", C.c_int, [H, C.c_int, P, P]),
    ("aao_rk_pint_apply", C.c_int, [H, P, P, C.c_int]),
    ("aao_rk_inner_solve", C.c_int, [H, C.c_int, P, P, C.POINTER(C.c_int)]),
    ("aao_rk_shifted_solve_noalloc", C.c_int, [C.POINTER(aao_grid), C.c_double, C.c_int, C.c_int, C.c_int,
                                               C.c_double, P, P, C.c_void_p]),
]


def load(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`"
                          " (there is no CPU fallback)")
    lib = C.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_LIB = None


def lib() -> C.CDLL:
    global _LIB
    if _LIB is None:
        _LIB = load()
    return _LIB


class AaoError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def check(status: int, allow=()) -> int:
    if status != AAO_OK and status not in allow:
        raise AaoError(status, lib().aao_rk_last_error().decode(errors="replace"))
    return status
