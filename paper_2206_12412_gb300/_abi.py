"""ctypes mirror of include/lbm.h, include/lbm_adjoint.h and
include/lbm_decomp.h (structs, constants, prototypes)."""
from __future__ import annotations

import ctypes as C

LBM_OK, LBM_ERR_ARG, LBM_ERR_CUDA, LBM_ERR_OOM = 0, -1, -2, -3
LBM_ERR_UNSTABLE, LBM_ERR_TIMEOUT, LBM_ERR_STATE, LBM_ERR_IO = -4, -5, -6, -7
STATUS_NAMES = {0: "LBM_OK", -1: "LBM_ERR_ARG", -2: "LBM_ERR_CUDA", -3: "LBM_ERR_OOM",
                -4: "LBM_ERR_UNSTABLE", -5: "LBM_ERR_TIMEOUT", -6: "LBM_ERR_STATE", -7: "LBM_ERR_IO"}

EDGE = {"free": 0, "dirichlet": 1, "periodic": 2}
EDGE_INDEX = {"left": 0, "right": 1, "bottom": 2, "top": 3}
STORAGE = {"f64": 0, "f32": 1, "f32_bf16": 2, "f32_f16": 3, "f32_lf": 4}
BC = {"bounceback": 0, "macroscopic": 1, "macroscopic_edges": 2}
VELOCITY_SET = {"D2Q5": 0, "D2Q9": 1}
CRACK = {"none": 0, "stationary": 1, "prescribed": 2, "kcrit": 3}
LOAD = {"zero": 0, "linear": 1, "sin2": 2, "halfsine": 3, "series": 4, "const": 5}
FIELD = {"w": 0, "wdot": 1}
MASK = {"h": 0, "v": 1}
FLAG_CLAMPED, FLAG_NONFINITE = 1, 4


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("dh", C.c_double), ("dt", C.c_double),
                ("edge", C.c_int32 * 4)]


class Lattice_(C.Structure):
    _fields_ = [("velocity_set", C.c_int32), ("form", C.c_int32), ("omega", C.c_double),
                ("storage", C.c_int32), ("bc_mode", C.c_int32)]


class Material(C.Structure):
    _fields_ = [("rho", C.c_double), ("mu", C.c_double)]


class Crack(C.Structure):
    _fields_ = [("mode", C.c_int32), ("two_tips", C.c_int32),
                ("y", C.c_double), ("x_start", C.c_double), ("x_tip", C.c_double),
                ("v_rel", C.c_double), ("K_C", C.c_double), ("v_max", C.c_double),
                ("r0", C.c_double), ("r_min", C.c_double), ("fit_width", C.c_double),
                ("hist_cap", C.c_int64)]


class CrackLine(C.Structure):
    _fields_ = [("mode", C.c_int32), ("two_tips", C.c_int32),
                ("x_start", C.c_double), ("y_start", C.c_double), ("x_tip", C.c_double), ("y_tip", C.c_double),
                ("v_rel", C.c_double), ("K_C", C.c_double), ("v_max", C.c_double),
                ("r0", C.c_double), ("r_min", C.c_double), ("fit_width", C.c_double),
                ("hist_cap", C.c_int64)]


class Loading(C.Structure):
    _fields_ = [("edge", C.c_int32), ("kind", C.c_int32), ("amp", C.c_double), ("t_ramp", C.c_double),
                ("series", C.POINTER(C.c_double)), ("n_series", C.c_int64)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
RELEASE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("release", RELEASE_FN), ("ctx", C.c_void_p)]


class CrackStateT(C.Structure):
    _fields_ = [("step", C.c_int64), ("tip_q", C.c_int64), ("n_cut", C.c_int64), ("hist_n", C.c_int64),
                ("tip_x", C.c_double), ("K", C.c_double), ("v", C.c_double), ("r_min", C.c_double),
                ("npairs", C.c_int32), ("flags", C.c_int32)]


# name -> (restype, argtypes); every symbol include/lbm.h declares
PROTOTYPES = {
    "lbm_create": (C.c_int, [C.POINTER(Grid), C.POINTER(Lattice_), C.POINTER(Material), C.POINTER(Crack),
                             C.POINTER(Loading), C.c_int32, C.c_void_p, C.POINTER(Allocator),
                             C.POINTER(C.c_void_p)]),
    "lbm_create_line": (C.c_int, [C.POINTER(Grid), C.POINTER(Lattice_), C.POINTER(Material), C.POINTER(CrackLine),
                                  C.POINTER(Loading), C.c_int32, C.c_void_p, C.POINTER(Allocator),
                                  C.POINTER(C.c_void_p)]),
    "lbm_line_tip": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                               C.c_int64, C.POINTER(C.c_int64)]),
    "lbm_line_tip_left": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                    C.c_int64, C.POINTER(C.c_int64)]),
    "lbm_step": (C.c_int, [C.c_void_p, C.c_int64]),
    "lbm_fields": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_int32]),
    "lbm_set_fields": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_int32]),
    "lbm_fields_strided": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_int32, C.c_int64]),
    "lbm_set_fields_strided": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_int32, C.c_int64]),
    "lbm_cut_mask": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_uint32), C.c_int64]),
    "lbm_crack_state": (C.c_int, [C.c_void_p, C.POINTER(CrackStateT), C.POINTER(C.c_double),
                                  C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                  C.c_int64, C.POINTER(C.c_int64)]),
    "lbm_crack_state_left": (C.c_int, [C.c_void_p, C.POINTER(CrackStateT), C.POINTER(C.c_double),
                                       C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                       C.c_int64, C.POINTER(C.c_int64)]),
    "lbm_sync": (C.c_int, [C.c_void_p]),
    "lbm_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lbm_set_launch": (C.c_int, [C.c_void_p, C.c_int32]),
    "lbm_get_launch": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                 C.POINTER(C.c_int32)]),
    "lbm_set_profiling": (C.c_int, [C.c_void_p, C.c_int32]),
    "lbm_profile_read": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_double),
                                   C.POINTER(C.c_int64), C.c_int32]),
    "lbm_set_wd_scale": (C.c_int, [C.c_void_p, C.c_double]),
    "lbm_get_wd_scale": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "lbm_device_bytes": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "lbm_save": (C.c_int, [C.c_void_p, C.c_char_p]),
    "lbm_load": (C.c_int, [C.c_void_p, C.c_char_p]),
    "lbm_destroy": (None, [C.c_void_p]),
    "lbm_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.c_int32, C.POINTER(Allocator),
                                   C.POINTER(C.c_void_p)]),
    "lbm_batch_step": (C.c_int, [C.c_void_p, C.c_int64]),
    "lbm_create_batch": (C.c_int, [C.c_int32, C.POINTER(Grid), C.POINTER(Lattice_), C.POINTER(Material),
                                   C.POINTER(Crack), C.POINTER(C.POINTER(Loading)), C.POINTER(C.c_int32),
                                   C.c_void_p, C.POINTER(Allocator), C.c_int32, C.POINTER(C.c_void_p)]),
    "lbm_batch_member": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_void_p)]),
    "lbm_batch_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "lbm_set_face_solve": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32)]),
    "lbm_set_bulk": (C.c_int, [C.c_void_p, C.c_int32]),
    "lbm_set_chained": (C.c_int, [C.c_void_p, C.c_int32]),
    "lbm_batch_set_chained": (C.c_int, [C.c_void_p, C.c_int32]),
    "lbm_batch_set_shape": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32]),
    "lbm_batch_set_persistent": (C.c_int, [C.c_void_p, C.c_int32, C.c_int64]),
    "lbm_barrier_probe": (C.c_int, [C.c_int32, C.c_int32, C.c_int64, C.c_void_p]),
    "lbm_batch_get_shape": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "lbm_batch_set_lookahead": (C.c_int, [C.c_void_p, C.c_int32]),
    "lbm_batch_get_lookahead": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32)]),
    "lbm_batch_tune": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                 C.POINTER(C.c_double), C.POINTER(C.c_int32)]),
    "lbm_batch_destroy": (None, [C.c_void_p]),
    "lbm_reset": (C.c_int, [C.c_void_p]),
    "lbm_wdot_to_host_noalloc": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.c_int64]),
    "lbm_set_loading": (C.c_int, [C.c_void_p, C.POINTER(Loading)]),
    "lbm_last_error": (C.c_char_p, []),
    # include/lbm_adjoint.h
    "lbm_tape_create": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.c_int32, C.c_int64, C.c_int32,
                                  C.POINTER(Allocator), C.POINTER(C.c_void_p)]),
    "lbm_tape_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(C.c_double)]),
    "lbm_tape_loss_device": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p)]),
    "lbm_tape_backward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32,
                                    C.c_int32]),
    "lbm_tape_misfits": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "lbm_tape_destroy": (None, [C.c_void_p]),
    "lbm_adjoint": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.c_int32, C.c_int64, C.c_int32, C.c_void_p,
                              C.c_int32, C.POINTER(C.c_double), C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                              C.c_int32, C.c_int32, C.POINTER(Allocator)]),
    # include/lbm_decomp.h
    "lbm_decomp_plan": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_int32)]),
    "lbm_decomp_create": (C.c_int, [C.POINTER(Grid), C.POINTER(Lattice_), C.POINTER(Material), C.POINTER(Crack),
                                    C.POINTER(Loading), C.c_int32, C.c_int32, C.POINTER(C.c_int32), C.c_void_p,
                                    C.POINTER(Allocator), C.POINTER(C.c_void_p)]),
    "lbm_decomp_step": (C.c_int, [C.c_void_p, C.c_int64]),
    "lbm_decomp_fields": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_int32]),
    "lbm_decomp_set_fields": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_int32]),
    "lbm_decomp_rank": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_void_p), C.POINTER(C.c_int32),
                                  C.POINTER(C.c_int32)]),
    "lbm_decomp_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "lbm_decomp_destroy": (None, [C.c_void_p]),
    "lbm_slab_create": (C.c_int, [C.POINTER(Grid), C.POINTER(Lattice_), C.POINTER(Material), C.POINTER(Crack),
                                  C.POINTER(Loading), C.c_int32, C.c_int32, C.c_int32, C.c_void_p,
                                  C.POINTER(Allocator), C.POINTER(C.c_void_p)]),
    "lbm_slab_export": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32]),
    "lbm_slab_import": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32]),
}
