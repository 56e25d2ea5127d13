"""ctypes declarations of the structure and coupling entry points (include/kbc_lbm.h)."""
from __future__ import annotations

import ctypes


class fem_beam_config(ctypes.Structure):
    _fields_ = [
        ("nn", ctypes.c_int),
        ("X", ctypes.c_void_p),
        ("EA", ctypes.c_double), ("EI", ctypes.c_double), ("rhoA", ctypes.c_double),
        ("thickness", ctypes.c_double),
        ("fixed", ctypes.c_void_p),
        ("theta", ctypes.c_double), ("lambda_", ctypes.c_double),
        ("rtol", ctypes.c_double), ("atol", ctypes.c_double),
        ("max_it", ctypes.c_int),
        ("dt", ctypes.c_double),
        ("stream", ctypes.c_void_p),
    ]


def declare(L):
    vp, i32, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
    L.fem_beam_workspace_size.argtypes = [ctypes.POINTER(fem_beam_config), ctypes.POINTER(sz)]
    L.fem_beam_create.argtypes = [ctypes.POINTER(fem_beam_config), vp, sz, ctypes.POINTER(vp)]
    L.fem_beam_step.argtypes = [vp, vp]
    L.fem_beam_get_state.argtypes = [vp, vp, vp, vp]
    L.fem_beam_set_state.argtypes = [vp, vp, vp, vp]
    L.fem_last_error.argtypes = [vp]
    L.fem_last_error.restype = ctypes.c_char_p
    L.fem_destroy.argtypes = [vp]
    L.fem_destroy.restype = None
    L.fsi_couple.argtypes = [vp, vp, i32]
    for name in ("fem_beam_workspace_size", "fem_beam_create", "fem_beam_step", "fem_beam_get_state",
                 "fem_beam_set_state", "fsi_couple"):
        getattr(L, name).restype = ctypes.c_int
