"""ctypes declarations of the C ABI in include/cfet.h (argument marshalling only)."""

from __future__ import annotations

import ctypes as C
import os

from . import build as _build

c_double_p = C.POINTER(C.c_double)
c_int32_p = C.POINTER(C.c_int32)
c_int64_p = C.POINTER(C.c_int64)

CFET_OK, CFET_EINVAL, CFET_ENOMEM, CFET_ECUDA, CFET_EKRYLOV, CFET_ETIMEOUT, CFET_ENAN, CFET_ENODEV = range(8)
STATUS_NAMES = ["CFET_OK", "CFET_EINVAL", "CFET_ENOMEM", "CFET_ECUDA", "CFET_EKRYLOV", "CFET_ETIMEOUT",
                "CFET_ENAN", "CFET_ENODEV"]
CFET_OP_XXZ_CHAIN, CFET_OP_X_FIELD, CFET_OP_DIA, CFET_OP_PAULI, CFET_OP_CSR = 1, 2, 3, 4, 5
c_uint64_p = C.POINTER(C.c_uint64)

SCHEME_IDS = {"CF2:1": 1, "CF4:2": 2, "CF4:3": 3, "CF4:3Opt": 4, "CF6:4": 5, "CF6:5": 6, "CF6:5b": 7,
              "CF6:6": 8, "CF6:5Imp": 9, "CF6:5Opt": 10, "CF6:6Opt": 11, "CF8:11": 12}


class cfet_op(C.Structure):
    _fields_ = [("kind", C.c_int32), ("nsites", C.c_int32), ("dim", C.c_int64), ("J", C.c_double),
                ("Delta", C.c_double), ("site_coeff", c_double_p), ("ndiag", C.c_int32),
                ("offsets", c_int64_p), ("values", c_double_p), ("nterms", C.c_int32),
                ("xmask", c_uint64_p), ("zmask", c_uint64_p), ("coeff", c_double_p),
                ("row_ptr", c_int64_p), ("col_idx", c_int32_p), ("csr_re", c_double_p), ("csr_im", c_double_p)]


class cfet_options(C.Structure):
    _fields_ = [("m_max", C.c_int32), ("m_min", C.c_int32), ("max_substeps", C.c_int32),
                ("block_size", C.c_int32), ("grid_size", C.c_int32), ("steps_per_launch", C.c_int32),
                ("barrier_timeout_s", C.c_double), ("precision", C.c_int32), ("expm", C.c_int32),
                ("picture", C.c_int32), ("reorth", C.c_int32),
                ("apply_form", C.c_int32)]


CFET_PREC_DEFAULT, CFET_PREC_F64, CFET_PREC_FX, CFET_PREC_C64 = 0, 1, 2, 3
PRECISIONS = {"default": CFET_PREC_DEFAULT, "f64": CFET_PREC_F64, "fx": CFET_PREC_FX, "c64": CFET_PREC_C64}
CFET_EXPM_KRYLOV, CFET_EXPM_CHEBYSHEV = 0, 1
EXPM = {"krylov": CFET_EXPM_KRYLOV, "chebyshev": CFET_EXPM_CHEBYSHEV}
CFET_PICTURE_SCHROEDINGER, CFET_PICTURE_INTERACTION = 0, 1
PICTURES = {"schroedinger": CFET_PICTURE_SCHROEDINGER, "interaction": CFET_PICTURE_INTERACTION}
CFET_APPLY_AUTO, CFET_APPLY_ELEMENTWISE, CFET_APPLY_TILED = 0, 1, 2
APPLY_FORMS = {"auto": CFET_APPLY_AUTO, "elementwise": CFET_APPLY_ELEMENTWISE, "tiled": CFET_APPLY_TILED}


class cfet_stats(C.Structure):
    _fields_ = [("n_exp", C.c_int64), ("n_substeps", C.c_int64), ("n_applies", C.c_int64),
                ("max_k", C.c_int32), ("status", C.c_int32), ("max_err_est", C.c_double),
                ("phase_ns", C.c_int64 * 8), ("phase_max_ns", C.c_int64 * 8)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if not f.startswith("phase")}
        d["phase_ns"] = list(self.phase_ns)
        d["phase_max_ns"] = list(self.phase_max_ns)
        return d

class cfet_decisions(C.Structure):
    _fields_ = [("n_exp", C.c_int64), ("n_sub", c_int32_p), ("k", c_int32_p), ("h", c_int32_p),
                ("cap", C.c_int64), ("len", C.c_int64)]


DRIVE_FN = C.CFUNCTYPE(C.c_double, C.c_double, C.c_void_p)


class cfet_grad_stats(C.Structure):
    _fields_ = [("overlap_re", C.c_double), ("overlap_im", C.c_double), ("max_drift", C.c_double),
                ("n_applies_forward", C.c_int64), ("n_applies_backward", C.c_int64), ("forward_ms", C.c_float),
                ("backward_ms", C.c_float)]


class cfet_chain(C.Structure):
    _fields_ = [("nsites", C.c_int32), ("J", C.c_double), ("Delta", C.c_double), ("h", c_double_p),
                ("a", c_double_p), ("f", DRIVE_FN), ("user", C.c_void_p), ("A", C.c_double),
                ("omega", C.c_double), ("phase", C.c_double)]


class cfet_batch_plan(C.Structure):
    _fields_ = [("cluster_size", C.c_int32), ("threads", C.c_int32), ("coop_min_sites", C.c_int32),
                ("tuned_ms", C.c_float)]

_lib = None


def library_path() -> str:
    return _build.LIB_PATH


def load() -> C.CDLL:
    """Load the compiled library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing: run paper_1102_5071_gb300.build.build() first")
    lib = C.CDLL(path)
    vp = C.c_void_p
    sigs = {
        "cfet_options_default": (None, [C.POINTER(cfet_options)]),
        "cfet_scheme_info": (C.c_int, [C.c_int32, c_int32_p, c_int32_p, c_int32_p, c_double_p, c_double_p,
                                       c_double_p, c_double_p, C.c_int32]),
        "cfet_chebyshev_coefficients": (C.c_int, [C.c_double, C.c_double, C.c_int32, c_double_p, c_int32_p,
                                                  c_double_p]),
        "cfet_create": (C.c_int, [C.POINTER(vp), C.POINTER(cfet_op), C.c_int32, C.POINTER(cfet_op),
                                  C.POINTER(DRIVE_FN), C.POINTER(vp), C.POINTER(cfet_options)]),
        "cfet_destroy": (None, [vp]),
        "cfet_last_error": (C.c_char_p, [vp]),
        "cfet_apply": (C.c_int, [vp, c_double_p, vp, vp, vp]),
        "cfet_expv": (C.c_int, [vp, c_double_p, C.c_double, vp, C.c_double, vp, C.POINTER(cfet_stats)]),
        "cfet_propagate": (C.c_int, [vp, vp, C.c_double, C.c_double, C.c_int64, C.c_int32, C.c_double, vp,
                                     C.POINTER(cfet_stats)]),
        "cfet_propagate_ex": (C.c_int, [vp, vp, C.c_double, C.c_double, C.c_int64, C.c_int32, C.c_int32,
                                        C.c_double, vp, C.POINTER(cfet_decisions), C.POINTER(cfet_decisions),
                                        C.POINTER(cfet_stats)]),
        "cfet_propagate_host": (C.c_int, [vp, vp, C.c_double, C.c_double, C.c_int64, C.c_int32, C.c_double, vp,
                                          C.POINTER(cfet_stats)]),
        "cfet_sync": (C.c_int, [vp, vp, C.POINTER(cfet_stats)]),
        "cfet_kernel_time_ms": (C.c_int, [vp, C.POINTER(C.c_float)]),
        "cfet_expv_chain_static": (C.c_int, [C.c_int32, C.c_double, C.c_double, c_double_p, c_double_p,
                                             C.c_double, C.c_double, C.c_double, vp, C.c_double, C.c_int32, vp,
                                             C.POINTER(cfet_stats)]),
        "cfet_batch_create": (C.c_int, [C.POINTER(vp), C.c_int32, C.POINTER(cfet_chain), C.POINTER(cfet_options)]),
        "cfet_batch_destroy": (None, [vp]),
        "cfet_batch_last_error": (C.c_char_p, [vp]),
        "cfet_batch_size": (C.c_int32, [vp]),
        "cfet_batch_propagate": (C.c_int, [vp, C.POINTER(vp), C.c_double, C.c_double, C.c_int64, C.c_int32,
                                           C.c_double, vp, C.POINTER(cfet_decisions), C.POINTER(cfet_decisions),
                                           C.POINTER(cfet_stats)]),
        "cfet_batch_tune": (C.c_int, [vp, C.c_double, C.c_double, C.c_int32, C.c_double, C.c_int64, vp,
                                      C.POINTER(cfet_batch_plan)]),
        "cfet_batch_get_plan": (C.c_int, [vp, C.POINTER(cfet_batch_plan)]),
        "cfet_batch_set_plan": (C.c_int, [vp, C.POINTER(cfet_batch_plan)]),
        "cfet_batch_kernel_time_ms": (C.c_int, [vp, C.POINTER(C.c_float)]),
        "cfet_fidelity_grad": (C.c_int, [vp, vp, vp, C.c_double, C.c_double, C.c_int64, C.c_int32, C.c_double,
                                         C.c_int32, c_double_p, C.c_double, C.c_double, C.c_int64, vp, c_double_p,
                                         c_double_p, C.POINTER(cfet_grad_stats)]),
        "cfet_selftest_wait_timeout": (C.c_int, [C.c_int32, C.c_double, c_int32_p]),
        "cfet_selftest_tiling": (C.c_int, [C.c_int32, C.c_int32, C.POINTER(C.c_int64)]),
        "cfet_selftest_i128_to_double": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p]),
        "cfet_selftest_ll_to_double_up": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p]),
        "cfet_selftest_krylov_bounds": (C.c_int, [C.c_int32, C.c_void_p, C.c_void_p, C.c_double,
                                                  C.c_void_p, C.POINTER(C.c_int32)]),
        "cfet_probe_copy_gbs": (C.c_int, [vp, vp, C.c_int64, C.c_int32, vp, c_double_p]),
        "cfet_error_constant": (C.c_int, [vp, vp, C.c_double, C.c_double, C.c_int64, C.c_int32, C.c_int32,
                                          C.c_double, C.c_double, vp, c_double_p, c_double_p, c_double_p]),
        "cfet_select_dt": (C.c_int, [vp, vp, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int64, C.c_int32,
                                     C.c_int32, C.c_double, C.c_double, vp, c_double_p, C.POINTER(C.c_int64),
                                     c_double_p]),
        "cfet_propagate_adaptive": (C.c_int, [vp, vp, C.c_double, C.c_double, C.c_int32, C.c_int32, C.c_double,
                                              C.c_double, C.c_double, C.c_double, C.c_double, C.c_int64, c_double_p,
                                              C.c_int64, c_double_p, C.c_int64, C.POINTER(C.c_int64),
                                              C.POINTER(C.c_int64), vp, C.POINTER(cfet_stats)]),
        "cfet_dim": (C.c_int64, [vp]),
        "cfet_num_drives": (C.c_int32, [vp]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


EXPORTED = ["cfet_options_default", "cfet_scheme_info", "cfet_chebyshev_coefficients", "cfet_create", "cfet_destroy", "cfet_last_error",
            "cfet_apply", "cfet_expv", "cfet_propagate", "cfet_propagate_ex", "cfet_propagate_host", "cfet_sync",
            "cfet_kernel_time_ms", "cfet_expv_chain_static",
            "cfet_batch_create", "cfet_batch_destroy", "cfet_batch_last_error", "cfet_batch_size",
            "cfet_batch_propagate", "cfet_batch_tune", "cfet_batch_get_plan", "cfet_batch_set_plan",
            "cfet_batch_kernel_time_ms", "cfet_fidelity_grad", "cfet_selftest_wait_timeout", "cfet_selftest_tiling",
            "cfet_selftest_i128_to_double", "cfet_selftest_ll_to_double_up", "cfet_selftest_krylov_bounds",
            "cfet_probe_copy_gbs", "cfet_error_constant", "cfet_select_dt", "cfet_propagate_adaptive",
            "cfet_dim", "cfet_num_drives"]
