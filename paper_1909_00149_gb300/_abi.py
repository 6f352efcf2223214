"""ctypes declarations of the C ABI in include/otprox.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libotprox.so")

OT_OK = 0
OT_EINVAL = -1
OT_ENOMEM = -2
OT_ECUDA = -3
OT_ENOTCONV = -4
OT_ENONFINITE = -5
OT_ETIMEOUT = -6
STATUS_NAMES = {0: "OT_OK", -1: "OT_EINVAL", -2: "OT_ENOMEM", -3: "OT_ECUDA", -4: "OT_ENOTCONV",
                -5: "OT_ENONFINITE", -6: "OT_ETIMEOUT"}

MODES = {"prox": 0, "fixed_first": 1, "eval": 2}
NORMS = {"iso": 0, "aniso": 1}
KERNELS = {"auto": 0, "tiled": 1, "resident": 2, "tma": 3, "temporal": 4}
PRECISIONS = {"fp32": 0, "split_bf16": 1, "split_bf16_3": 2}
ALGORITHMS = {"alg1": 0, "projection": 1}

c_float_p = ctypes.POINTER(ctypes.c_float)
c_double_p = ctypes.POINTER(ctypes.c_double)


class ot_prox_params(ctypes.Structure):
    _fields_ = [("B", ctypes.c_int32), ("H", ctypes.c_int32), ("W", ctypes.c_int32),
                ("mode", ctypes.c_int32), ("norm", ctypes.c_int32), ("balanced", ctypes.c_int32),
                ("p_exp", ctypes.c_int32),
                ("mu", ctypes.c_double), ("rho", ctypes.c_double),
                ("tau1", ctypes.c_double), ("tau2", ctypes.c_double), ("tol", ctypes.c_double),
                ("max_iter", ctypes.c_int32), ("check_every", ctypes.c_int32),
                ("kernel", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("algorithm", ctypes.c_int32), ("precision", ctypes.c_int32), ("beta", ctypes.c_double),
                ("tb_depth", ctypes.c_int32)]


class ot_prox_result(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("status", ctypes.c_int32),
                ("res_pri", ctypes.c_double), ("res_fp", ctypes.c_double),
                ("objective", ctypes.c_double), ("primal_feasible", ctypes.c_double),
                ("dual_obj", ctypes.c_double), ("rel_gap", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class ot_rpca_params(ctypes.Structure):
    _fields_ = [("T", ctypes.c_int32), ("H", ctypes.c_int32), ("W", ctypes.c_int32),
                ("lambda_", ctypes.c_double), ("gamma", ctypes.c_double), ("kappa", ctypes.c_double),
                ("mu", ctypes.c_double), ("rho", ctypes.c_double), ("n_inner", ctypes.c_int32),
                ("tol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("check_every", ctypes.c_int32),
                ("svt_max_sweeps", ctypes.c_int32), ("prox_kernel", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("signed_fg", ctypes.c_int32)]


class ot_rpca_result(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("status", ctypes.c_int32), ("res_pri", ctypes.c_double),
                ("res_dual", ctypes.c_double), ("svt_rounds", ctypes.c_int32), ("svt_rank", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class ot_prox_batch_result(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("status", ctypes.c_int32), ("res_pri", ctypes.c_double),
                ("res_fp", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class ot_uotdf_params(ctypes.Structure):
    _fields_ = [("B", ctypes.c_int32), ("H", ctypes.c_int32), ("W", ctypes.c_int32),
                ("kappa", ctypes.c_double), ("mu", ctypes.c_double), ("rho", ctypes.c_double),
                ("lambda_", ctypes.c_double), ("n_inner", ctypes.c_int32), ("norm", ctypes.c_int32),
                ("p_exp", ctypes.c_int32), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int32),
                ("check_every", ctypes.c_int32), ("prox_kernel", ctypes.c_int32)]


class ot_uotdf_result(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("status", ctypes.c_int32), ("res_pri", ctypes.c_double),
                ("res_dual", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


UOTDF_VARS = {"s": 0, "x": 1, "z": 2, "a": 3, "b": 4}

RPCA_VARS = {"S": 0, "L": 1, "X": 2, "T": 3, "A": 4, "D": 5, "B": 6, "C": 7, "Z": 8, "W": 9,
             "Mx": 10, "My": 11, "r": 12, "a": 13, "Sp": 14, "Sm": 15}
RPCA_PAIR_VARS = {"B", "C", "Z", "W", "Mx", "My", "r", "a"}
# signed foreground: a pair variable of the S- sign is its name with a "-"
# suffix ("Z-", "B-", ...), read with this flag on the variable id
RPCA_MINUS = 0x100
for _n in list(RPCA_PAIR_VARS):
    RPCA_VARS[_n + "-"] = RPCA_VARS[_n] | RPCA_MINUS
RPCA_PAIR_VARS |= {_n + "-" for _n in RPCA_PAIR_VARS}

# (name, restype, argtypes)
PROTOTYPES = [
    ("ot_last_error", ctypes.c_char_p, []),
    ("ot_prox_default_params", None, [ctypes.POINTER(ot_prox_params)]),
    ("ot_lambda_max", ctypes.c_double, [ctypes.c_int32, ctypes.c_int32]),
    ("ot_n_identity_blocks", ctypes.c_int32, [ctypes.c_int32, ctypes.c_int32]),
    ("ot_prox_create", ctypes.c_int, [ctypes.POINTER(ot_prox_params), ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    ("ot_prox_set_input", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("ot_prox_step", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    ("ot_prox_solve", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ot_prox_result)]),
    ("ot_prox_check_interval", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ot_prox_result)]),
    ("ot_prox_step_timed", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]),
    ("ot_prox_evaluate", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ot_prox_result)]),
    ("ot_prox_get_state", ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_void_p] * 6),
    ("ot_prox_set_state", ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_void_p] * 6),
    ("ot_prox_reset", ctypes.c_int, [ctypes.c_void_p]),
    ("ot_prox_get_params", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ot_prox_params)]),
    ("ot_prox_destroy", ctypes.c_int, [ctypes.c_void_p]),
    ("ot_rpca_default_params", None, [ctypes.POINTER(ot_rpca_params)]),
    ("ot_rpca_create", ctypes.c_int, [ctypes.POINTER(ot_rpca_params), ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    ("ot_rpca_set_input", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("ot_rpca_step", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    ("ot_rpca_iterate_checked", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ot_rpca_result)]),
    ("ot_rpca_solve", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ot_rpca_result)]),
    ("ot_rpca_get", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    ("ot_rpca_step_profiled", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    ("ot_debug_grid_barrier", ctypes.c_int, [ctypes.c_int32, ctypes.c_uint32, ctypes.POINTER(ctypes.c_int32),
                                             ctypes.POINTER(ctypes.c_uint32)]),
    ("ot_rpca_reset", ctypes.c_int, [ctypes.c_void_p]),
    ("ot_rpca_get_params", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ot_rpca_params)]),
    ("ot_rpca_destroy", ctypes.c_int, [ctypes.c_void_p]),
    ("ot_prox_batch_create", ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                            ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                            ctypes.POINTER(ot_prox_params), ctypes.c_void_p,
                                            ctypes.POINTER(ctypes.c_void_p)]),
    ("ot_prox_batch_set_input", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    ("ot_prox_batch_step", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    ("ot_prox_batch_solve", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ot_prox_batch_result),
                                           ctypes.POINTER(ctypes.c_int32)]),
    ("ot_prox_batch_get_state", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32] + [ctypes.c_void_p] * 6),
    ("ot_prox_batch_set_config", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    ("ot_prox_batch_autotune", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32),
                                              ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                              ctypes.POINTER(ctypes.c_float)]),
    ("ot_prox_batch_reset", ctypes.c_int, [ctypes.c_void_p]),
    ("ot_prox_batch_destroy", ctypes.c_int, [ctypes.c_void_p]),
    ("ot_uotdf_default_params", None, [ctypes.POINTER(ot_uotdf_params)]),
    ("ot_uotdf_create", ctypes.c_int, [ctypes.POINTER(ot_uotdf_params), ctypes.c_void_p,
                                       ctypes.POINTER(ctypes.c_void_p)]),
    ("ot_uotdf_set_input", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("ot_uotdf_step", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    ("ot_uotdf_iterate_checked", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ot_uotdf_result)]),
    ("ot_uotdf_solve", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ot_uotdf_result)]),
    ("ot_uotdf_get", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    ("ot_uotdf_reset", ctypes.c_int, [ctypes.c_void_p]),
    ("ot_uotdf_get_params", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ot_uotdf_params)]),
    ("ot_uotdf_destroy", ctypes.c_int, [ctypes.c_void_p]),
    ("ot_prox_warm_start", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double]),
    ("ot_unet_create", ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                      ctypes.POINTER(ctypes.c_void_p)]),
    ("ot_unet_param_count", ctypes.c_int64, [ctypes.c_void_p]),
    ("ot_unet_set_params", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("ot_unet_get_params", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("ot_unet_set_bias_free", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    ("ot_unet_forward", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]),
    ("ot_unet_gradients", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                         ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    ("ot_unet_train_step", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                          ctypes.c_float, ctypes.POINTER(ctypes.c_double)]),
    ("ot_unet_destroy", ctypes.c_int, [ctypes.c_void_p]),
    ("ot_svt", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double,
                              ctypes.c_void_p]),
    ("ot_neumann_solve", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_int32, ctypes.c_double, ctypes.c_int32, ctypes.c_void_p]),
    ("ot_neumann_solve_timed", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                               ctypes.c_int32, ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                               ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    ("ot_prox_evaluate_noalloc", ctypes.c_int, [ctypes.POINTER(ot_prox_params)] + [ctypes.c_void_p] * 8 +
     [ctypes.POINTER(ot_prox_result), ctypes.c_void_p]),
]


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libotprox.so and declare its prototypes.  Raises if it is absent:
    there is no fallback implementation."""
    if not os.path.exists(path):
        raise ImportError(f"libotprox.so is not built ({path}); run __graft_entry__.build() "
                          "or python -m paper_1909_00149_gb300.build")
    lib = ctypes.CDLL(path)
    for name, res, args in PROTOTYPES:
        if hasattr(lib, name):
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
    return lib
