"""ctypes declarations of include/esbgk.h (argument marshalling only).

Every function here forwards to libesbgk.so under the same name; all the
arithmetic runs in the library's CUDA kernels.  Importing this module fails
loudly when the library has not been built: there is no fallback.
"""

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libesbgk.so")

OK = 0
E_ARG, E_WORKSPACE, E_CUDA, E_NONREALIZABLE, E_TIMEOUT, E_STATE, E_TOO_LARGE = -1, -2, -3, -4, -5, -6, -7
STATUS_NAMES = {0: "OK", -1: "E_ARG", -2: "E_WORKSPACE", -3: "E_CUDA", -4: "E_NONREALIZABLE",
                -5: "E_TIMEOUT", -6: "E_STATE", -7: "E_TOO_LARGE"}
FP64, FP32, BF16 = 0, 1, 2
BC = {"periodic": 0, "outflow": 1}
SWITCH = {"frozen": 0, "plain": 1, "learned": 2}
CNN_PARAMS, CNN_CHANNELS = 10753, 16
COUPLING = {"stage": 0, "step": 1}
INTERFACE = {"own": 0, "conservative": 1}
TAU_MODEL = {"constant": 0, "density": 1}
PREC = {"fp64": FP64, "fp32": FP32, "bf16": BF16}
KERNEL_CLASSES = ("l1", "flags", "compact", "prep", "stage", "final", "other")


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("x0", ctypes.c_double),
                ("x1", ctypes.c_double), ("y0", ctypes.c_double), ("y1", ctypes.c_double),
                ("bc_x", ctypes.c_int32), ("bc_y", ctypes.c_int32)]


class VMesh(ctypes.Structure):
    _fields_ = [("nv", ctypes.c_int32), ("vmax", ctypes.c_double)]


class Params(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("tau", ctypes.c_double), ("eta_factor", ctypes.c_double),
                ("delta", ctypes.c_double), ("cweno_eps", ctypes.c_double), ("sw", ctypes.c_int32),
                ("coupling", ctypes.c_int32), ("prec", ctypes.c_int32), ("interface_flux", ctypes.c_int32),
                ("tau_model", ctypes.c_int32), ("moment_sums", ctypes.c_int32)]


class Tableau(ctypes.Structure):
    _fields_ = [("s", ctypes.c_int32), ("At", ctypes.c_double * 16), ("bt", ctypes.c_double * 4),
                ("A", ctypes.c_double * 16), ("b", ctypes.c_double * 4)]


class Error(RuntimeError):
    def __init__(self, code, msg="", bad_cell=-1):
        self.code = code
        self.bad_cell = bad_cell
        super().__init__("%s (%d): %s" % (STATUS_NAMES.get(code, "?"), code, msg))


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            "libesbgk.so is not built (%s). Build it with `python -m paper_2512_03586_gb300.build` "
            "(nvcc for sm_103a); there is no CPU fallback." % LIB_PATH)
    return ctypes.CDLL(LIB_PATH)


lib = _load()

P = ctypes.c_void_p
D = ctypes.POINTER(ctypes.c_double)
U8 = ctypes.POINTER(ctypes.c_uint8)
I = ctypes.c_int
LL = ctypes.POINTER(ctypes.c_longlong)

_SIGS = {
    "esbgk_version": (I, []),
    "esbgk_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(Grid), ctypes.POINTER(VMesh), ctypes.POINTER(Params)]),
    "esbgk_create": (I, [ctypes.POINTER(Grid), ctypes.POINTER(VMesh), ctypes.POINTER(Params), P, ctypes.c_size_t,
                         P, ctypes.POINTER(P)]),
    "esbgk_destroy": (None, [P]),
    "esbgk_set_state": (I, [P, D, D, D, D, D, U8]),
    "esbgk_set_f": (I, [P, D]),
    "esbgk_get_f": (I, [P, D]),
    "esbgk_regime_update": (I, [P]),
    "esbgk_set_flags": (I, [P, U8]),
    "esbgk_get_flags": (I, [P, U8]),
    "esbgk_get_indicators": (I, [P, D, D]),
    "esbgk_advance": (I, [P, ctypes.c_double, ctypes.POINTER(Tableau)]),
    "esbgk_step": (I, [P, ctypes.c_double, ctypes.POINTER(Tableau)]),
    "esbgk_get_moments": (I, [P, D, D, D, D]),
    "esbgk_get_cons": (I, [P, D]),
    "esbgk_totals": (I, [P, D]),
    "esbgk_counters": (I, [P, LL, LL, LL, LL]),
    "esbgk_graphs": (I, [P, ctypes.c_int32]),
    "esbgk_kinetic_form": (I, [P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "esbgk_tiles": (I, [P, ctypes.c_int32]),
    "esbgk_set_solid": (I, [P, ctypes.c_void_p]),
    "esbgk_tiled": (I, [P, ctypes.POINTER(ctypes.c_int32)]),
    "esbgk_wait_probe": (I, [ctypes.c_int32, ctypes.c_int32, P]),
    "esbgk_timing": (I, [P, I]),
    "esbgk_timing_read": (I, [P, D, LL, ctypes.c_int32]),
    "esbgk_sync": (I, [P]),
    "esbgk_last_error": (I, [P, ctypes.c_char_p, ctypes.c_size_t, LL]),
    "esbgk_relax_cells": (I, [P, D, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                              ctypes.c_int32, P, P, P]),
    "esbgk_batch_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int32, ctypes.POINTER(Grid), ctypes.POINTER(VMesh),
                                                      ctypes.POINTER(Params)]),
    "esbgk_batch_create": (I, [ctypes.c_int32, ctypes.POINTER(Grid), ctypes.POINTER(VMesh), ctypes.POINTER(Params),
                               P, ctypes.c_size_t, P, ctypes.POINTER(P)]),
    "esbgk_batch_destroy": (None, [P]),
    "esbgk_batch_set_state": (I, [P, ctypes.c_int32, D, D, D, D, D, U8]),
    "esbgk_batch_step": (I, [P, D, ctypes.POINTER(Tableau), ctypes.c_int32]),
    "esbgk_batch_get_moments": (I, [P, ctypes.c_int32, D, D, D, D]),
    "esbgk_batch_get_cons": (I, [P, ctypes.c_int32, D]),
    "esbgk_batch_get_flags": (I, [P, ctypes.c_int32, U8]),
    "esbgk_batch_counters": (I, [P, LL, LL, LL, LL]),
    "esbgk_batch_autotune": (I, [P, D, ctypes.POINTER(Tableau), ctypes.POINTER(ctypes.c_int32),
                                 ctypes.POINTER(ctypes.c_int32)]),
    "esbgk_batch_schedule": (I, [P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                 ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32), ctypes.c_int32,
                                 ctypes.POINTER(ctypes.c_int32)]),
    "esbgk_batch_set_form": (I, [P, ctypes.c_int32, ctypes.c_int32]),
    "esbgk_batch_set_switch_params": (I, [P, ctypes.c_int32, ctypes.POINTER(ctypes.c_float)]),
    "esbgk_batch_switch_stats": (I, [P, ctypes.c_int32, LL, LL, LL, LL]),
    "esbgk_batch_sync": (I, [P]),
    "esbgk_batch_timing": (I, [P, ctypes.c_int32]),
    "esbgk_batch_timing_read": (I, [P, D, LL, ctypes.c_int32]),
    "esbgk_batch_last_error": (I, [P, ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_int32)]),
    "esbgk_set_switch_params": (I, [P, ctypes.POINTER(ctypes.c_float)]),
    "esbgk_switch_stats": (I, [P, LL, LL, LL, LL]),
    "esbgk_features": (I, [P, P]),
    "esbgk_cnn_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    "esbgk_cnn_create": (I, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P, ctypes.c_size_t, P,
                             ctypes.POINTER(P)]),
    "esbgk_cnn_destroy": (None, [P]),
    "esbgk_cnn_set_params": (I, [P, ctypes.POINTER(ctypes.c_float)]),
    "esbgk_cnn_get_params": (I, [P, ctypes.POINTER(ctypes.c_float)]),
    "esbgk_cnn_forward": (I, [P, P, ctypes.c_int32, P]),
    "esbgk_cnn_gradient": (I, [P, P, P, ctypes.c_int32, ctypes.c_float, ctypes.POINTER(ctypes.c_float),
                               ctypes.POINTER(ctypes.c_float)]),
    "esbgk_cnn_train_step": (I, [P, P, P, ctypes.c_int32, ctypes.c_float, ctypes.c_float,
                                 ctypes.POINTER(ctypes.c_float)]),
    "esbgk_cnn_sync": (I, [P]),
    "esbgk_kinetic_steps_noalloc": (I, [ctypes.POINTER(Grid), ctypes.POINTER(VMesh), ctypes.POINTER(Params),
                                        ctypes.c_double, ctypes.POINTER(Tableau), ctypes.c_int32, D, P, D, P]),
}

for _name, (_res, _args) in _SIGS.items():
    _fn = getattr(lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args
    globals()[_name] = _fn

DECLARED = tuple(_SIGS)
