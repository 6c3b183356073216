"""ctypes binding of libftsp2.so: the C ABI of include/ftsp2.h, function for
function, plus the struct layouts.  Argument marshalling only; every step of
the hot path runs in the library's CUDA kernels.  Importing this module fails
loudly when the library has not been built (there is no fallback)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libftsp2.so")

# status codes
OK, E_ARG, E_CUDA, E_WORKSPACE, E_VALIDITY, E_NONFINITE, E_TIMEOUT, E_NOMODEL, E_UNSUPPORTED = \
    0, -1, -2, -3, -4, -5, -6, -7, -8
# modes
FP32, TF32X3, BF16X3, FP16X2 = 0, 1, 2, 3
MODES = {"fp32": FP32, "tf32x3": TF32X3, "bf16x3": BF16X3, "fp16x2": FP16X2}
# flags
SYNC, CLAMP, REFINE1, REFINE2, PAIR_TILES, SINGLE_TILES, LANCZOS, MIN_LAYERS, REFINE_TC = \
    0x1, 0x2, 0x4, 0x8, 0x10, 0x20, 0x40, 0x80, 0x100
EPI_DEFERRED, EPI_INLINE, FULL_OPERANDS = 0x200, 0x400, 0x800
LAYER_LAUNCHES = 0x1000
FAMILY_MLSP2, FAMILY_SKIP, FAMILY_MAX = 0, 1, 2
TARGET_FERMI, TARGET_ENTROPY = 0, 1


class Instance(C.Structure):
    _fields_ = [("n", C.c_int32), ("reserved", C.c_int32), ("offset", C.c_int64),
                ("mu", C.c_double), ("kT", C.c_double)]


class Table(C.Structure):
    _fields_ = [("L", C.c_int32), ("L_entropy", C.c_int32), ("beta0", C.c_double),
                ("mu0", C.c_double), ("alpha", C.c_double),
                ("theta", C.POINTER(C.c_double)), ("theta_entropy", C.POINTER(C.c_double)),
                ("family", C.c_int32), ("reserved", C.c_int32)]


class RescaleRec(C.Structure):
    _fields_ = [("e_min", C.c_double), ("e_max", C.c_double), ("mu_p", C.c_double),
                ("beta_p", C.c_double), ("scale", C.c_double), ("flip", C.c_int32),
                ("model", C.c_int32), ("status", C.c_int32), ("layers", C.c_int32),
                ("valid", C.c_int32), ("reserved", C.c_int32)]


class TrainReport(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("accepted", C.c_int32), ("cost0", C.c_double),
                ("cost", C.c_double), ("max_err", C.c_double), ("lam", C.c_double)]


assert C.sizeof(Instance) == 32 and C.sizeof(RescaleRec) == 64

# every function the header declares, with its signature
_VP, _SZ, _I, _D = C.c_void_p, C.c_size_t, C.c_int, C.c_double
_PINST = C.POINTER(Instance)
SIGNATURES = {
    "ftsp2_model_set_create": (_I, [C.POINTER(Table), _I, C.POINTER(_VP)]),
    "ftsp2_model_set_builtin": (_I, [C.POINTER(_VP)]),
    "ftsp2_model_set_destroy": (None, [_VP]),
    "ftsp2_model_set_info": (_I, [_VP, C.POINTER(_I), C.POINTER(_I)]),
    "ftsp2_model_set_table": (_I, [_VP, _I, C.POINTER(_I), C.POINTER(_D), C.POINTER(_D), C.POINTER(_D),
                                   C.POINTER(_D)]),
    "ftsp2_workspace_size": (_I, [_PINST, _I, _I, _I, C.POINTER(_SZ)]),
    "ftsp2_workspace_size_set": (_I, [_PINST, _I, _VP, _I, _I, C.POINTER(_SZ)]),
    "ftsp2_rescale_workspace_size": (_I, [_I, C.POINTER(_SZ)]),
    "ftsp2_rescale": (_I, [_VP, _PINST, _VP, _I, _VP, _I, _VP, _VP, _SZ, _VP]),
    "ftsp2_density": (_I, [_VP, _PINST, _VP, _I, _VP, _I, _I, _VP, _VP, _VP, _VP, _SZ, _VP]),
    "ftsp2_entropy": (_I, [_VP, _PINST, _VP, _I, _VP, _I, _I, _VP, _VP, _VP, _SZ, _VP]),
    "ftsp2_density_entropy": (_I, [_VP, _PINST, _VP, _I, _VP, _I, _I, _VP, _VP, _VP, _VP, _VP, _SZ, _VP]),
    "ftsp2_density_noalloc": (_I, [_VP, _PINST, _VP, _I, _VP, _I, _I, _VP, _VP, _VP, _VP]),
    "ftsp2_density_mu": (_I, [_VP, _PINST, _VP, _I, _VP, _VP, _I, _I, _I, _D, _VP, _VP, _VP, _VP, _VP, _VP, _SZ,
                              _VP]),
    "ftsp2_autotune": (_I, [_VP, _PINST, _VP, _I, _VP, _I, _I, _VP, _VP, _VP, _VP, _VP, _SZ, _I,
                            C.POINTER(_I), C.POINTER(C.c_float), _VP]),
    "ftsp2_tile_shape": (_I, [_PINST, _I, _I, _I, _I, C.POINTER(_I), C.POINTER(_I)]),
    "ftsp2_autotune_clear": (_I, []),
    "ftsp2_train_workspace_size": (_SZ, [_I, _I]),
    "ftsp2_train_coeffs": (_I, [_I, _D, _D, _I, _D, _I, C.c_uint64, _I, _I, C.POINTER(_D), C.POINTER(_D),
                                C.POINTER(TrainReport), _VP, _SZ, _VP]),
    "ftsp2_train_coeffs_alt": (_I, [_I, _D, _D, _I, _D, _I, C.c_uint64, _I, _I, C.POINTER(_D), C.POINTER(_D),
                                    C.POINTER(TrainReport), _VP, _SZ, _VP]),
    "ftsp2_alt_to_mlsp2": (_I, [_I, C.POINTER(_D), C.POINTER(_D)]),
    "ftsp2_train_coeffs_skip": (_I, [_I, _D, _D, _I, _D, _I, C.c_uint64, _I, _I, C.POINTER(_D), C.POINTER(_D),
                                     C.POINTER(TrainReport), _VP, _SZ, _VP]),
    "ftsp2_train_workspace_size_max": (_SZ, [_I, _I]),
    "ftsp2_train_coeffs_max": (_I, [_I, _D, _D, _I, _D, _I, C.c_uint64, _I, _I, C.POINTER(_D), C.POINTER(_D),
                                    C.POINTER(TrainReport), _VP, _SZ, _VP]),
    "ftsp2_train_coeffs_skipk": (_I, [_I, _D, _D, _I, _I, _I, _D, _I, C.c_uint64, _I, _I, C.POINTER(_D),
                                      C.POINTER(_D), C.POINTER(TrainReport), _VP, _SZ, _VP]),
    "ftsp2_train_init_skipk": (_I, [_I, _I, _I, _D, _D, C.POINTER(_D)]),
    "ftsp2_skipk_to_max": (_I, [_I, _I, _I, C.POINTER(_D), C.POINTER(_D)]),
    "ftsp2_train_samples": (_I, [_D, _D, _I, C.c_uint64, C.POINTER(_D)]),
    "ftsp2_train_init": (_I, [_I, _D, _D, C.POINTER(_D)]),
    "ftsp2_train_init_alt": (_I, [_I, _D, C.POINTER(_D)]),
    "ftsp2_mlsp2_to_skip": (_I, [_I, C.POINTER(_D), C.POINTER(_D)]),
    "ftsp2_mlsp2_to_max": (_I, [_I, C.POINTER(_D), C.POINTER(_D)]),
    "ftsp2_skip_to_max": (_I, [_I, _I, _I, C.POINTER(_D), C.POINTER(_D), C.POINTER(_D), C.POINTER(_D), _D,
                               C.POINTER(_D)]),
    "ftsp2_layer_count": (_D, [_D]),
    "ftsp2_train_residuals": (_I, [_I, _I, _D, _D, _I, _D, C.POINTER(_D), _VP, _I, _VP, _VP]),
    "ftsp2_train_residual_jacobian": (_I, [_I, _D, _D, _I, _D, C.POINTER(_D), _VP, _I, _VP, _VP, _VP]),
    "ftsp2_train_normal_equations": (_I, [_VP, _I, _I, _VP, _VP, _SZ, _VP]),
    "ftsp2_profile_layers": (_I, [_I]),
    "ftsp2_profile_read": (_I, [C.POINTER(_D), C.POINTER(C.c_uint64)]),
    "ftsp2_status_string": (C.c_char_p, [_I]),
    "ftsp2_kernel_launch_count": (C.c_uint64, []),
    "ftsp2_set_wait_limit_ns": (_I, [C.c_uint64]),
    "ftsp2_wait_limit_ns": (C.c_uint64, []),
    "ftsp2_debug_stall_layer": (_I, [_I]),
}

_lib = None


def lib():
    """The loaded library.  Raises if libftsp2.so is missing: there is no CPU path."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libftsp2.so is not built; run paper_2605_08523_gb300.build.build() "
                               "(the hot path has no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def status_string(s: int) -> str:
    return lib().ftsp2_status_string(s).decode()


class Ftsp2Error(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__("%s failed: %s (%d)" % (where, status_string(code), code))
        self.code = code


def check(code: int, where: str):
    if code != OK:
        raise Ftsp2Error(code, where)
    return code
