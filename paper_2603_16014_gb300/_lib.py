"""ctypes loader for libmtgp_gb300.so (the C ABI declared in include/mtgp.h).

Argument marshalling only.  Loading fails loudly when the library has not been built: there is
no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmtgp_gb300.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "mtgp.h")

MTGP_OK = 0
ERRORS = {
    1: "MTGP_ERR_INVALID_ARG", 2: "MTGP_ERR_NOT_PD", 3: "MTGP_ERR_NUMERIC", 4: "MTGP_ERR_TIMEOUT",
    5: "MTGP_ERR_UNSUPPORTED", 6: "MTGP_ERR_CUDA", 7: "MTGP_ERR_STATE",
}
LATTICE, DNET = 0, 1
FP64, FP32_TRANSFORM = 0, 1
NOISE_PER_TASK = 16
SOLVE_FP64 = 32

_p = ctypes.c_void_p
_i = ctypes.c_int
_SIGS = {
    "mtgp_create": (_i, [ctypes.POINTER(_p), _i, _i, _i, _p, _p, _i, _p, _i]),
    "mtgp_destroy": (_i, [_p]),
    "mtgp_points": (_i, [_p, _p, _p]),
    "mtgp_set_y": (_i, [_p, _p, _p]),
    "mtgp_nll": (_i, [_p, _p, _p, _i, _p, _p, _p, _p, _p]),
    "mtgp_nll_grad": (_i, [_p, _p, _p, _i, _p, _p, _p, _p, _p, _p, _p, _p, _p]),
    "mtgp_posterior": (_i, [_p, _p, _p, _i, _p, _p, _i, _p, _p, _p, _p, _p]),
    "mtgp_sync": (_i, [_p, _p]),
    "mtgp_last_error_string": (ctypes.c_char_p, []),
    "mtgp_workspace_bytes": (ctypes.c_longlong, [_p]),
    "mtgp_profile": (_i, [_p, _i]),
    "mtgp_profile_read": (_i, [_p, _i, _p, _p, _p, _p]),
    "mtgp_nll_equal_static": (_i, [_i, _i, _i, _i, _p, _i, _p, _i, _p, _p, _p, _i, _p, _p, _p, _p, _p, _p]),
    "mtgp_batch_create": (_i, [ctypes.POINTER(_p), _i, _p, _p, _p, _p, _p, _p, _p, _i, _p]),
    "mtgp_batch_destroy": (_i, [_p]),
    "mtgp_batch_layout": (_i, [_p, _p, _p]),
    "mtgp_batch_set_y": (_i, [_p, _p, _p]),
    "mtgp_batch_set_theta": (_i, [_p, _p, _p]),
    "mtgp_batch_get_theta": (_i, [_p, _p, _p]),
    "mtgp_batch_nll_grad": (_i, [_p, _p, _p, _p]),
    "mtgp_batch_adam": (_i, [_p, _i, ctypes.c_double, _i, _p, _p]),
    "mtgp_batch_autotune": (_i, [_p, _i, _p, _p]),
    "mtgp_batch_fit": (_i, [_p, _p, _i, ctypes.c_double, _i, _p, _p, _p, _p]),
    "mtgp_propose": (_i, [_p, _p, _p, _i, _p, _p]),
    "mtgp_selftest_arith": (_i, [_i, ctypes.c_longlong, _p, _p, _p, _p]),
    "mtgp_gcv": (_i, [_p, _p, _p, _i, _p, _p, _p, _p, _p]),
    "mtgp_set_smoothness": (_i, [_p, _i]),
    "mtgp_set_dsi_weights": (_i, [_p, _p, _p]),
    "mtgp_nll_grad_host": (_i, [_p, _p, _i, _p, _p]),
    "mtgp_dsi_weights_grad": (_i, [_p, _p, _p]),
    "mtgp_cubature": (_i, [_p, _p, _p, _i, _p, _p, _p, _p, _p]),
    "mtgp_gcv_grad": (_i, [_p, _p, _p, _i, _p, _p, _p, _p, _p, _p, _p, _p, _p]),
    "mtgp_batch_features": (_i, [_p, _p, _p]),
    "mtgp_batch_targets": (_i, [_p, _p, _p, _p]),
    "mtgp_batch_set_theta_proposal": (_i, [_p, _p, _p]),
    "mtgp_mlp_create": (_i, [ctypes.POINTER(_p), _i, _p, _i]),
    "mtgp_mlp_destroy": (_i, [_p]),
    "mtgp_mlp_set_params": (_i, [_p, _p, _p, _p]),
    "mtgp_mlp_get_params": (_i, [_p, _p, _p, _p]),
    "mtgp_mlp_fit_scaling": (_i, [_p, _i, _p, _p]),
    "mtgp_mlp_forward": (_i, [_p, _i, _p, _p, _p]),
    "mtgp_mlp_gradients": (_i, [_p, _i, _p, _p, _p, _p, _p, _p, _p]),
    "mtgp_mlp_train_step": (_i, [_p, _i, _p, _p, _p, _p, ctypes.c_float, _p, _p]),
}

_LIB = None


class MTGPError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {ERRORS.get(code, code)}: {msg}")
        self.code = code


def declared_symbols() -> list:
    """Function names declared in include/mtgp.h."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"\b(mtgp_[a-z_]+)\s*\(", txt)))


def lib() -> ctypes.CDLL:
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2603_16014_gb300.build.build() "
                               "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def check(code: int, where: str) -> None:
    if code != MTGP_OK:
        msg = lib().mtgp_last_error_string()
        raise MTGPError(code, where, msg.decode() if msg else "")
