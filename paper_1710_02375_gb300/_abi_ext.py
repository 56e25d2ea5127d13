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
        ("solve_fp64", ctypes.c_int),
    ]


class fem_shell_config(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("X", ctypes.c_void_p),
        ("E", ctypes.c_double), ("nu", ctypes.c_double), ("h", ctypes.c_double),
        ("rho", ctypes.c_double),
        ("fixed", ctypes.c_void_p),
        ("theta", ctypes.c_double), ("lambda_", ctypes.c_double),
        ("rtol", ctypes.c_double), ("atol", ctypes.c_double),
        ("max_it", ctypes.c_int),
        ("dt", ctypes.c_double),
        ("max_cg", ctypes.c_int),
        ("cg_rtol", ctypes.c_double),
        ("stream", ctypes.c_void_p),
    ]


class fem_svk_config(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("nn", ctypes.c_int), ("ne", ctypes.c_int),
        ("X", ctypes.c_void_p), ("conn", ctypes.c_void_p), ("fixed", ctypes.c_void_p),
        ("E", ctypes.c_double), ("nu", ctypes.c_double), ("rho", ctypes.c_double),
        ("theta", ctypes.c_double), ("lambda_", ctypes.c_double),
        ("rtol", ctypes.c_double), ("atol", ctypes.c_double),
        ("max_it", ctypes.c_int),
        ("dt", ctypes.c_double),
        ("max_cg", ctypes.c_int),
        ("cg_rtol", ctypes.c_double),
        ("stream", ctypes.c_void_p),
        ("solve_fp64", ctypes.c_int),
    ]


class mlp_config(ctypes.Structure):
    _fields_ = [
        ("n_layers", ctypes.c_int),
        ("dims", ctypes.c_int * 9),
        ("max_batch", ctypes.c_int),
        ("lr", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
        ("eps", ctypes.c_double),
        ("stream", ctypes.c_void_p),
    ]


class lbm_multiphase_params(ctypes.Structure):
    _fields_ = [
        ("kappa", ctypes.c_double),
        ("eos", ctypes.c_int),
        ("g", ctypes.c_double * 3),
        ("kappa_w", ctypes.c_double),
    ]


def declare(L):
    vp, i32, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
    L.lbm_set_multiphase.argtypes = [vp, ctypes.POINTER(lbm_multiphase_params)]
    L.lbm_set_multiphase.restype = ctypes.c_int
    L.lbm_get_force_field.argtypes = [vp, vp]
    L.lbm_refine_workspace_size.argtypes = [vp, vp, ctypes.POINTER(sz)]
    L.lbm_refine_couple.argtypes = [vp, vp, i32, i32, vp, sz]
    L.lbm_get_force_field.restype = ctypes.c_int
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
    L.fsi_couple_span.argtypes = [vp, vp, i32, i32, ctypes.c_double, ctypes.c_double]
    L.fsi_couple_span.restype = ctypes.c_int
    L.fsi_couple_shell.argtypes = [vp, vp, i32]
    L.fsi_couple_shell.restype = ctypes.c_int
    L.fem_shell_workspace_size.argtypes = [ctypes.POINTER(fem_shell_config), ctypes.POINTER(sz)]
    L.fem_shell_create.argtypes = [ctypes.POINTER(fem_shell_config), vp, sz, ctypes.POINTER(vp)]
    L.fem_shell_step.argtypes = [vp, vp]
    L.fem_shell_get_state.argtypes = [vp, vp, vp, vp, vp]
    L.fem_shell_set_state.argtypes = [vp, vp, vp, vp, vp]
    L.fem_shell_last_error.argtypes = [vp]
    L.fem_shell_last_error.restype = ctypes.c_char_p
    L.fem_shell_destroy.argtypes = [vp]
    L.fem_shell_destroy.restype = None
    for name in ("fem_shell_workspace_size", "fem_shell_create", "fem_shell_step",
                 "fem_shell_get_state", "fem_shell_set_state"):
        getattr(L, name).restype = ctypes.c_int
    L.fem_svk_workspace_size.argtypes = [ctypes.POINTER(fem_svk_config), ctypes.POINTER(sz)]
    L.fem_svk_create.argtypes = [ctypes.POINTER(fem_svk_config), vp, sz, ctypes.POINTER(vp)]
    L.fem_svk_step.argtypes = [vp, vp]
    L.fem_svk_body_load.argtypes = [vp, vp, vp]
    L.fem_svk_get_state.argtypes = [vp, vp, vp, vp]
    L.fem_svk_set_state.argtypes = [vp, vp, vp, vp]
    L.fem_svk_last_error.argtypes = [vp]
    L.fem_svk_last_error.restype = ctypes.c_char_p
    L.fem_svk_destroy.argtypes = [vp]
    L.fem_svk_destroy.restype = None
    for name in ("fem_svk_workspace_size", "fem_svk_create", "fem_svk_step", "fem_svk_body_load",
                 "fem_svk_get_state", "fem_svk_set_state"):
        getattr(L, name).restype = ctypes.c_int
    L.lbm_batch_workspace_size.argtypes = [vp, i32, ctypes.POINTER(sz)]
    L.lbm_batch_create.argtypes = [vp, i32, vp, sz, ctypes.POINTER(vp)]
    L.lbm_batch_step.argtypes = [vp, i32]
    L.lbm_batch_step_graph.argtypes = [vp, i32, i32]
    L.lbm_batch_set_tuning.argtypes = [vp, i32, i32]
    L.lbm_batch_autotune.argtypes = [vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                     ctypes.POINTER(ctypes.c_float)]
    L.lbm_batch_last_error.argtypes = [vp]
    L.lbm_batch_last_error.restype = ctypes.c_char_p
    L.lbm_batch_destroy.argtypes = [vp]
    L.lbm_batch_destroy.restype = None
    L.mlp_workspace_size.argtypes = [ctypes.POINTER(mlp_config), ctypes.POINTER(sz)]
    L.mlp_create.argtypes = [ctypes.POINTER(mlp_config), vp, sz, ctypes.POINTER(vp)]
    L.mlp_set_params.argtypes = [vp, vp]
    L.mlp_get_params.argtypes = [vp, vp]
    L.mlp_param_count.argtypes = [vp]
    L.mlp_param_count.restype = ctypes.c_longlong
    L.mlp_forward.argtypes = [vp, vp, i32, vp]
    L.mlp_gradients.argtypes = [vp, vp, vp, i32, vp, vp]
    L.mlp_train_step.argtypes = [vp, vp, vp, i32, vp]
    L.mlp_set_learning_rate.argtypes = [vp, ctypes.c_double]
    L.mlp_set_learning_rate.restype = ctypes.c_int
    L.mlp_last_error.argtypes = [vp]
    L.mlp_last_error.restype = ctypes.c_char_p
    L.mlp_destroy.argtypes = [vp]
    L.mlp_destroy.restype = None
    for name in ("mlp_workspace_size", "mlp_create", "mlp_set_params", "mlp_get_params", "mlp_forward",
                 "mlp_gradients", "mlp_train_step"):
        getattr(L, name).restype = ctypes.c_int
    for name in ("lbm_batch_workspace_size", "lbm_batch_create", "lbm_batch_step",
                 "lbm_batch_step_graph", "lbm_batch_set_tuning", "lbm_batch_autotune"):
        getattr(L, name).restype = ctypes.c_int
    for name in ("fem_beam_workspace_size", "fem_beam_create", "fem_beam_step", "fem_beam_get_state",
                 "fem_beam_set_state", "fsi_couple"):
        getattr(L, name).restype = ctypes.c_int
