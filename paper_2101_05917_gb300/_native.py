"""ctypes binding of libdiffpd.so (argument marshalling only).

Every entry point declared in include/diffpd.h is bound here under the same
name.  The library must have been built (paper_2101_05917_gb300.build.build());
there is no fallback: a missing library raises.
"""
from __future__ import annotations

import ctypes
import os

from .build import LIB

PD_OK = 0
PD_ERR_INVALID_ARG = 1
PD_ERR_OOM = 2
PD_ERR_NOT_SPD = 3
PD_ERR_NOT_CONVERGED = 4
PD_ERR_INVERTED = 5
PD_ERR_NAN = 6
PD_ERR_TIMEOUT = 7
PD_ERR_CUDA = 8
PD_ERR_NO_DEVICE = 9
PD_ERR_INTERNAL = 10
STATUS_NAMES = {0: "PD_OK", 1: "PD_ERR_INVALID_ARG", 2: "PD_ERR_OOM", 3: "PD_ERR_NOT_SPD",
                4: "PD_ERR_NOT_CONVERGED", 5: "PD_ERR_INVERTED", 6: "PD_ERR_NAN",
                7: "PD_ERR_TIMEOUT", 8: "PD_ERR_CUDA", 9: "PD_ERR_NO_DEVICE",
                10: "PD_ERR_INTERNAL"}

PD_PREC_FP64 = 0
PD_PREC_MIXED = 1
PD_PREC_MIXED_STRAIN = 2
PD_PREC_FP64_REFINED = 3
PD_ELEM_HEX8 = 0
PD_ELEM_TET6 = 1
PD_ELEM_TETU = 2   # unstructured tetrahedra: pd_create_tet_mesh only
ELEMENT_RULES = {"hex8": PD_ELEM_HEX8, "tet6": PD_ELEM_TET6}

EXPORT = {"inc_ptr": 0, "inc": 1, "perm": 2, "snode_first": 3, "row_ptr": 4, "rows": 5, "parent": 6,
          "level": 7, "rel": 8, "level_ptr": 9, "level_list": 10, "solve_tiles": 11}

c_double_p = ctypes.POINTER(ctypes.c_double)
c_u8_p = ctypes.POINTER(ctypes.c_uint8)
c_i64_p = ctypes.POINTER(ctypes.c_int64)


class MeshDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("dx", ctypes.c_double), ("origin", ctypes.c_double * 3), ("density", ctypes.c_double),
                ("cell_mask", c_u8_p), ("dirichlet", c_u8_p), ("contact", c_u8_p),
                ("leaf_max", ctypes.c_int32), ("device", ctypes.c_int32), ("element_rule", ctypes.c_int32)]


class TetMeshDesc(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("n_tets", ctypes.c_int64), ("X", c_double_p),
                ("tets", ctypes.POINTER(ctypes.c_int32)), ("density", ctypes.c_double),
                ("dirichlet", c_u8_p), ("contact", c_u8_p), ("leaf_max", ctypes.c_int32),
                ("device", ctypes.c_int32)]


class MeshInfo(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("n_elems", ctypes.c_int64), ("n_free", ctypes.c_int64),
                ("n_snodes", ctypes.c_int64), ("n_levels", ctypes.c_int64), ("factor_nnz", ctypes.c_int64),
                ("max_rows", ctypes.c_int64), ("max_cols", ctypes.c_int64),
                ("front_entries", ctypes.c_int64), ("update_entries", ctypes.c_int64),
                ("factorized", ctypes.c_int32), ("precision", ctypes.c_int32)]


class FactorOpts(ctypes.Structure):
    _fields_ = [("h", ctypes.c_double), ("gravity", ctypes.c_double * 3), ("k_contact", ctypes.c_double),
                ("precision", ctypes.c_int32), ("neohookean", ctypes.c_int32)]


class SolverOpts(ctypes.Structure):
    _fields_ = [("tol_fwd", ctypes.c_double), ("tol_bwd", ctypes.c_double),
                ("max_iter_fwd", ctypes.c_int32), ("max_iter_bwd", ctypes.c_int32),
                ("lbfgs_m", ctypes.c_int32), ("ls_max", ctypes.c_int32),
                ("checkpoint_every", ctypes.c_int32), ("check_every", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("warm_start", ctypes.c_int32),
                ("no_graphs", ctypes.c_int32), ("complementarity", ctypes.c_int32), ("step_ms", c_double_p),
                ("step_iters", ctypes.POINTER(ctypes.c_int32)), ("fext_per_step", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("fwd_iters", ctypes.c_int64), ("bwd_iters", ctypes.c_int64),
                ("fwd_fp64_iters", ctypes.c_int64), ("bwd_fp64_iters", ctypes.c_int64),
                ("fwd_line_search", ctypes.c_int64),
                ("max_fwd_iters_step", ctypes.c_int32), ("max_bwd_iters_step", ctypes.c_int32),
                ("max_fwd_rel_residual", ctypes.c_double), ("max_bwd_rel_residual", ctypes.c_double),
                ("inverted", ctypes.c_int32), ("not_converged_steps", ctypes.c_int32),
                ("fwd_ms", ctypes.c_double), ("bwd_ms", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64), ("solves", ctypes.c_int64), ("solve_ms", ctypes.c_double),
                ("local_steps", ctypes.c_int64), ("local_ms", ctypes.c_double),
                ("solves_timed", ctypes.c_int64), ("local_steps_timed", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Request(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("dx", ctypes.c_double), ("origin", ctypes.c_double * 3), ("density", ctypes.c_double),
                ("cell_mask_host", c_u8_p), ("dirichlet_host", c_u8_p), ("contact_host", c_u8_p),
                ("w_corot_host", c_double_p), ("w_vol_host", c_double_p), ("w_muscle_host", c_double_p),
                ("fiber_host", c_double_p), ("h", ctypes.c_double), ("gravity", ctypes.c_double * 3),
                ("k_contact", ctypes.c_double), ("mu", ctypes.c_double), ("precision", ctypes.c_int32),
                ("T", ctypes.c_int32), ("x0_host", c_double_p), ("v0_host", c_double_p),
                ("f_ext_host", c_double_p), ("act_host", c_double_p), ("loss_w_host", c_double_p),
                ("opts", SolverOpts)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("loss", ctypes.c_double), ("n_nodes", ctypes.c_int64),
                ("n_elems", ctypes.c_int64), ("T", ctypes.c_int64), ("x_final_host", c_double_p),
                ("g_v0_host", c_double_p), ("g_act_host", c_double_p), ("queue_ms", ctypes.c_double),
                ("latency_ms", ctypes.c_double), ("fwd_iters", ctypes.c_int64), ("bwd_iters", ctypes.c_int64),
                ("slot", ctypes.c_int32), ("mesh_cached", ctypes.c_int32), ("factor_cached", ctypes.c_int32)]


SYMBOLS = ["pd_create_mesh", "pd_create_tet_mesh", "pd_mesh_destroy", "pd_mesh_query", "pd_mesh_export", "pd_factorize",
           "pd_forward", "pd_backward", "pd_plan_checkpoints", "pd_local_step", "pd_hessian_vector", "pd_solve_A",
           "pd_local_step_noalloc", "pd_contact_prepare", "pd_contact_set", "pd_solve_A_contact", "pd_contact_step_set", "pd_serve_create", "pd_serve_submit", "pd_serve_poll", "pd_serve_release", "pd_serve_drain",
           "pd_serve_destroy", "pd_last_error"]

_lib = None


def lib() -> ctypes.CDLL:
    """Loads libdiffpd.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        raise RuntimeError(f"{LIB} is missing: build it with paper_2101_05917_gb300.build.build()")
    L = ctypes.CDLL(LIB)
    vp = ctypes.c_void_p
    st = ctypes.c_int32
    L.pd_create_mesh.argtypes = [ctypes.POINTER(MeshDesc), ctypes.POINTER(vp)]
    L.pd_create_mesh.restype = st
    L.pd_create_tet_mesh.argtypes = [ctypes.POINTER(TetMeshDesc), ctypes.POINTER(vp)]
    L.pd_create_tet_mesh.restype = st
    L.pd_mesh_destroy.argtypes = [vp]
    L.pd_mesh_destroy.restype = None
    L.pd_mesh_query.argtypes = [vp, ctypes.POINTER(MeshInfo)]
    L.pd_mesh_query.restype = st
    L.pd_mesh_export.argtypes = [vp, ctypes.c_int32, c_i64_p, ctypes.c_int64, c_i64_p]
    L.pd_mesh_export.restype = st
    L.pd_factorize.argtypes = [vp, vp, vp, vp, vp, ctypes.POINTER(FactorOpts), vp]
    L.pd_factorize.restype = st
    L.pd_forward.argtypes = [vp, vp, vp, vp, vp, ctypes.c_double, ctypes.c_int32, ctypes.POINTER(SolverOpts),
                             vp, vp, ctypes.POINTER(Stats), vp]
    L.pd_forward.restype = st
    L.pd_backward.argtypes = [vp, vp, vp, vp, vp, ctypes.c_double, ctypes.c_int32, vp, vp, ctypes.c_int32,
                              ctypes.POINTER(SolverOpts), vp, vp, vp, vp, vp, vp, vp, vp,
                              ctypes.POINTER(Stats), vp]
    L.pd_backward.restype = st
    L.pd_plan_checkpoints.argtypes = [vp, ctypes.c_int32, ctypes.c_size_t, ctypes.POINTER(ctypes.c_int32)]
    L.pd_plan_checkpoints.restype = st
    L.pd_local_step.argtypes = [vp, vp, vp, ctypes.c_int32, vp, vp, vp]
    L.pd_local_step.restype = st
    L.pd_hessian_vector.argtypes = [vp, vp, vp, vp, ctypes.c_int32, vp, vp]
    L.pd_hessian_vector.restype = st
    L.pd_solve_A.argtypes = [vp, vp, vp, ctypes.c_int32, vp]
    L.pd_solve_A.restype = st
    L.pd_local_step_noalloc.argtypes = [ctypes.c_int64, ctypes.c_int64, vp, vp, vp, ctypes.c_double, vp, vp, vp,
                                        vp, vp, vp, vp, ctypes.c_double, ctypes.c_int32, vp, vp, vp, vp]
    L.pd_local_step_noalloc.restype = st
    L.pd_serve_create.argtypes = [ctypes.c_int32, ctypes.c_size_t, ctypes.c_int32, ctypes.POINTER(vp)]
    L.pd_serve_create.restype = st
    L.pd_serve_submit.argtypes = [vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]
    L.pd_serve_submit.restype = st
    L.pd_serve_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(Result)]
    L.pd_serve_poll.restype = st
    L.pd_contact_prepare.argtypes = [vp, c_u8_p, vp]
    L.pd_contact_prepare.restype = st
    L.pd_contact_set.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), ctypes.c_int64, vp]
    L.pd_contact_set.restype = st
    L.pd_solve_A_contact.argtypes = [vp, vp, vp, vp, ctypes.c_int32, vp]
    L.pd_solve_A_contact.restype = st
    L.pd_contact_step_set.argtypes = [vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), c_u8_p, ctypes.c_int64,
                                      ctypes.POINTER(ctypes.c_int64)]
    L.pd_contact_step_set.restype = st
    L.pd_serve_release.argtypes = [vp, ctypes.c_uint64]
    L.pd_serve_release.restype = st
    L.pd_serve_drain.argtypes = [vp]
    L.pd_serve_drain.restype = st
    L.pd_serve_destroy.argtypes = [vp]
    L.pd_serve_destroy.restype = None
    L.pd_last_error.argtypes = []
    L.pd_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


class PDError(RuntimeError):
    def __init__(self, status, where):
        msg = lib().pd_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status, where, allow=()):
    if status != PD_OK and status not in allow:
        raise PDError(status, where)
    return status
