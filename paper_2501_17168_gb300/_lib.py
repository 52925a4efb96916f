"""ctypes binding of ``libtgp.so`` (the C ABI of ``include/tgp.h``).

Argument marshalling only.  The functions keep the C names and take the C
structures; every step of the computation runs in the library's kernels.
Loading fails loudly when the library has not been built -- there is no
other implementation to fall back to.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libtgp.so")

TGP_OK, TGP_ERR_INVALID_ARG, TGP_ERR_INVALID_TREE, TGP_ERR_WORKSPACE, TGP_ERR_CUDA, \
    TGP_ERR_TIMEOUT, TGP_ERR_UNSUPPORTED = range(7)
TREE_LEN, TREE_TYPE, TREE_FUNC, TREE_VAR, TREE_MODI, TREE_CONST, TREE_SIZE, TREE_DEPTH = \
    1, 2, 4, 8, 16, 32, 64, 128
TREE_NO_ADJOINT = 256
MAX_LEN, MAX_OUTPUTS, MAX_FEATURES = 1024, 16, 256
NOALLOC_WS_BYTES = 32 << 20
PICK_NODES, PICK_RANDOM, PICK_HOIST = 0, 1, 2
XCHG_TOO_LARGE, XCHG_DONE, XCHG_SKIPPED, XCHG_BAD_INDEX, XCHG_BAD_TREE = 0, 1, 2, -1, -2


class tgp_population(ctypes.Structure):
    _fields_ = [("type", ctypes.c_void_p), ("value", ctypes.c_void_p), ("size", ctypes.c_void_p),
                ("pop", ctypes.c_int64), ("max_len", ctypes.c_int32), ("ld", ctypes.c_int64)]


class tgp_data(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("n_points", ctypes.c_int64),
                ("n_features", ctypes.c_int32), ("ldx", ctypes.c_int64)]


class tgp_config(ctypes.Structure):
    _fields_ = [("trees_per_block", ctypes.c_int32), ("points_per_tile", ctypes.c_int32),
                ("tiles_per_item", ctypes.c_int32), ("points_per_lane", ctypes.c_int32),
                ("eval_begin_event", ctypes.c_void_p), ("eval_end_event", ctypes.c_void_p),
                ("flags", ctypes.c_int32), ("max_wait_polls", ctypes.c_int32),
                ("cta_width", ctypes.c_int32)]


FLAG_SSE = 1


class tgp_problem(ctypes.Structure):
    _fields_ = [("pop", tgp_population), ("data", tgp_data), ("y", ctypes.c_void_p),
                ("n_outputs", ctypes.c_int32), ("mse", ctypes.c_void_p),
                ("tree_status", ctypes.c_void_p), ("cfg", tgp_config)]


MAX_PROBLEMS = 16

_P = ctypes.POINTER
_lock = threading.Lock()
_lib = None

# name -> (restype, argtypes)
_SIGS = {
    "tgp_workspace_size": (ctypes.c_size_t, [_P(tgp_population), _P(tgp_data), ctypes.c_int32,
                                             _P(tgp_config)]),
    "tgp_validate": (ctypes.c_int, [_P(tgp_population), ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                    ctypes.c_void_p]),
    "tgp_eval_forward": (ctypes.c_int, [_P(tgp_population), _P(tgp_data), ctypes.c_int32,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_size_t, ctypes.c_void_p]),
    "tgp_eval_forward_cfg": (ctypes.c_int, [_P(tgp_population), _P(tgp_data), ctypes.c_int32,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_size_t, ctypes.c_void_p, _P(tgp_config)]),
    "tgp_fitness_mse": (ctypes.c_int, [_P(tgp_population), _P(tgp_data), ctypes.c_void_p,
                                       ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "tgp_fitness_mse_cfg": (ctypes.c_int, [_P(tgp_population), _P(tgp_data), ctypes.c_void_p,
                                           ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                           _P(tgp_config)]),
    "tgp_batch_workspace_size": (ctypes.c_size_t, [_P(tgp_problem), ctypes.c_int32]),
    "tgp_batch_fitness_mse": (ctypes.c_int, [_P(tgp_problem), ctypes.c_int32, ctypes.c_void_p,
                                             ctypes.c_size_t, ctypes.c_void_p]),
    "tgp_eval_backward": (ctypes.c_int, [_P(tgp_population), _P(tgp_data), ctypes.c_void_p,
                                         ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "tgp_eval_backward_cfg": (ctypes.c_int, [_P(tgp_population), _P(tgp_data), ctypes.c_void_p,
                                             ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                             _P(tgp_config)]),
    "tgp_fitness_mse_noalloc": (ctypes.c_int, [_P(tgp_population), _P(tgp_data), ctypes.c_void_p,
                                               ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_void_p]),
    "tgp_subtree_exchange": (ctypes.c_int, [_P(tgp_population), _P(tgp_population),
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32,
                                            ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]),
    "tgp_tournament_select": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                             ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                             ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "tgp_accuracy_from_outputs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                                 ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                                 ctypes.c_void_p, ctypes.c_void_p]),
    "tgp_accuracy_workspace_size": (ctypes.c_size_t, [_P(tgp_population), _P(tgp_data),
                                                      ctypes.c_int32]),
    "tgp_fitness_accuracy": (ctypes.c_int, [_P(tgp_population), _P(tgp_data), ctypes.c_void_p,
                                            ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                            ctypes.c_void_p]),
    "tgp_batch_plan": (ctypes.c_int, [_P(tgp_problem), ctypes.c_int32, ctypes.c_char_p,
                                      _P(ctypes.c_void_p)]),
    "tgp_batch_plan_workspace_size": (ctypes.c_size_t, [ctypes.c_void_p]),
    "tgp_tune_cache_lookup": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_char_p, _P(tgp_config)]),
    "tgp_batch_plan_shape": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, _P(tgp_config),
                                            _P(ctypes.c_int32)]),
    "tgp_batch_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                     ctypes.c_void_p]),
    "tgp_batch_free": (None, [ctypes.c_void_p]),
    "tgp_check_device_error": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "tgp_check_device_error_noalloc": (ctypes.c_int, [ctypes.c_void_p]),
    "tgp_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "tgp_version": (ctypes.c_char_p, []),
}


def load(path: str | None = None):
    """Loads the library (once) and declares every exported signature."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(
                    f"{p} is missing: build the CUDA library first "
                    "(python -m paper_2501_17168_gb300.build); there is no CPU fallback")
            lib = ctypes.CDLL(p)
            for name, (res, args) in _SIGS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def declared_symbols():
    return list(_SIGS)


class TGPError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        try:
            name = load().tgp_status_string(code).decode()
        except Exception:  # library not loadable: report the number
            name = str(code)
        super().__init__(f"{where} returned {name}")


def check(code: int, where: str):
    if code != TGP_OK:
        raise TGPError(code, where)
