"""ctypes binding of libelm.so (include/elm.h): argument marshalling only."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libelm.so")

ELM_OK, ELM_ERR_ARG, ELM_ERR_CUDA, ELM_ERR_TOPOLOGY = 0, 1, 2, 3
ELM_ERR_WALK_LIMIT, ELM_ERR_NONFINITE, ELM_ERR_STATE, ELM_ERR_NOT_CONVERGED = 4, 5, 6, 7
ELM_FP64, ELM_FP32 = 0, 1
STATUS_NAMES = {0: "ELM_OK", 1: "ELM_ERR_ARG", 2: "ELM_ERR_CUDA", 3: "ELM_ERR_TOPOLOGY",
                4: "ELM_ERR_WALK_LIMIT", 5: "ELM_ERR_NONFINITE", 6: "ELM_ERR_STATE", 7: "ELM_ERR_NOT_CONVERGED"}

# (name, restype, argtypes) of every entry point declared in include/elm.h
_P, _I64, _I, _D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
SIGNATURES = [
    ("elm_mesh_create", _I, [_I, _I64, _P, _I64, _P, _I, _I, ctypes.POINTER(_P)]),
    ("elm_mesh_destroy", _I, [_P]),
    ("elm_mesh_num_nodes", _I64, [_P]),
    ("elm_mesh_num_unique", _I64, [_P]),
    ("elm_mesh_set_annulus", _I, [_P, _D, _D, _I, _D]),
    ("elm_mesh_node_coords", _I, [_P, _P]),
    ("elm_mesh_unique_map", _I, [_P, _P]),
    ("elm_to_storage", _I, [_P, _P, _P, _I, _P]),
    ("elm_to_unique", _I, [_P, _P, _P, _I, _P]),
    ("elm_set_velocity", _I, [_P, _P, _P, _P]),
    ("elm_shift_velocity", _I, [_P, _P, _P]),
    ("elm_advect", _I, [_P, _P, _P, _D, _I, _P]),
    ("elm_advect_noalloc", _I, [_P, _P, _P, _P, _P, _D, _I, _P]),
    ("elm_advect_host", _I, [_P, _P, _P, _P, _P, _D, _I, _P]),
    ("elm_advect_adjoint", _I, [_P, _P, _P, _P, _P, _P, _D, _I, _P]),
    ("elm_trace", _I, [_P, _P, _P, _D, _I, _P]),
    ("elm_trace_eval", _I, [_P, _P, _P, _P, _P]),
    ("elm_diffusion_step", _I, [_P, _P, _P, _P, _P, _D, _D, _D, _D, _I, ctypes.POINTER(_I),
                                ctypes.POINTER(_D), _P]),
    ("elm_get_status", _I, [_P, _P]),
    ("elm_batch_create", _I, [_P, _I, _I, _I, ctypes.POINTER(_P)]),
    ("elm_batch_destroy", _I, [_P]),
    ("elm_batch_num_items", _I64, [_P]),
    ("elm_batch_advect", _I, [_P, _P, _P, _P, _P, _P]),
    ("elm_probe_pipes", _I, [ctypes.POINTER(_D), _I, _P]),
    ("elm_last_error", ctypes.c_char_p, []),
]

_lib = None


class ElmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads libelm.so; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"libelm.so not built ({path}); run `python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(path)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def check(status: int) -> None:
    if status != ELM_OK:
        raise ElmError(status, load().elm_last_error().decode(errors="replace"))

ELM_HOST_ONLY = 0x100
ELM_ADJOINT = 0x200
ELM_P1 = 0x400
ELM_DIFFUSION = 0x800
ELM_HOST_STAGING = 0x1000
