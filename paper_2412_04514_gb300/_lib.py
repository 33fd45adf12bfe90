"""ctypes view of the C ABI in include/vt.h (libvt.so).

This module only declares the structs and signatures and loads the library.
There is no fallback: if the CUDA library cannot be built or loaded, every
entry point raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

VT_OK = 0
VT_ERR_INVALID_ARG = 1
VT_ERR_CUDA = 2
VT_ERR_CAPACITY = 3
VT_ERR_UNVALIDATED = 4
VT_ERR_DUPLICATE_POINTS = 5
VT_ERR_TIMEOUT = 6
VT_ERR_WORKSPACE = 7
VT_ERR_INTERNAL = 8

VT_FP64 = 0
VT_FP32_RECHECK = 1
VT_INDEX_ORIGINAL = 0
VT_INDEX_SORTED = 1
VT_EMIT_NBR = 1
VT_EMIT_VOL = 2
VT_EMIT_CEN = 4
VT_EMIT_M2 = 8
VT_EMIT_GEOM = 16
VT_MAX_PASSES = 16
VT_FLAG_STAGE_TIMES = 1
VT_FLAG_NO_SYNC = 2
VT_FLAG_PERIODIC = 4
VT_FLAG_FUSED = 8

STATUS_NAMES = {
    0: "VT_OK", 1: "VT_ERR_INVALID_ARG", 2: "VT_ERR_CUDA", 3: "VT_ERR_CAPACITY", 4: "VT_ERR_UNVALIDATED",
    5: "VT_ERR_DUPLICATE_POINTS", 6: "VT_ERR_TIMEOUT", 7: "VT_ERR_WORKSPACE", 8: "VT_ERR_INTERNAL",
}

# every entry point declared in include/vt.h
EXPORTS = [
    "vt_params_default", "vt_grid_resolution", "vt_workspace_size", "vt_grid_build", "vt_knn", "vt_clip_cells",
    "vt_emit", "vt_tessellate", "vt_read_status", "vt_last_error", "vt_launch_count", "vt_version",
    "vt_grid_build_static", "vt_moments_adjoint", "vt_probe_fma", "vt_batch_plan", "vt_batch_workspace_size",
    "vt_tessellate_batch", "vt_read_stats", "vt_cluster_index", "vt_cluster_class", "vt_tune_space_default",
    "vt_autotune_workspace_size", "vt_autotune", "vt_autotune_batch_workspace_size", "vt_autotune_batch",
    "vt_unvalidated_cells", "vt_lloyd_step",
]
VT_TUNE_CLASSES = 4
VT_TUNE_MAX_TRIED = 64


class VtParams(ctypes.Structure):
    _fields_ = [
        ("k0", ctypes.c_int),
        ("k_max", ctypes.c_int),
        ("grid_density", ctypes.c_float),
        ("grid_res", ctypes.c_int),
        ("threads_per_cell", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("emit", ctypes.c_int),
        ("index_space", ctypes.c_int),
        ("box_lo", ctypes.c_float * 3),
        ("box_hi", ctypes.c_float * 3),
        ("flags", ctypes.c_int),
    ]


class VtCellsOut(ctypes.Structure):
    _fields_ = [
        ("vol", ctypes.c_void_p),
        ("cen", ctypes.c_void_p),
        ("m2", ctypes.c_void_p),
        ("nbr_off", ctypes.c_void_p),
        ("nbr", ctypes.c_void_p),
        ("nbr_cap", ctypes.c_int64),
        ("vtx_off", ctypes.c_void_p),
        ("vtx", ctypes.c_void_p),
        ("vtx_cap", ctypes.c_int64),
        ("face_off", ctypes.c_void_p),
        ("face_nbr", ctypes.c_void_p),
        ("face_vtx_off", ctypes.c_void_p),
        ("face_vtx", ctypes.c_void_p),
        ("face_cap", ctypes.c_int64),
        ("face_vtx_cap", ctypes.c_int64),
        ("perm", ctypes.c_void_p),
        ("needed_nbr", ctypes.c_int64),
        ("needed_vtx", ctypes.c_int64),
        ("needed_face", ctypes.c_int64),
        ("needed_face_vtx", ctypes.c_int64),
    ]


class VtSetDesc(ctypes.Structure):
    _fields_ = [
        ("G", ctypes.c_int),
        ("lo", ctypes.c_float * 3),
        ("hi", ctypes.c_float * 3),
        ("scale", ctypes.c_float * 3),
        ("cw", ctypes.c_double * 3),
        ("margin", ctypes.c_double),
        ("cell_base", ctypes.c_int64),
        ("pt_begin", ctypes.c_int64),
        ("npts", ctypes.c_int64),
        ("periodic", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


class VtTuneSpace(ctypes.Structure):
    _fields_ = [
        ("n_tpc", ctypes.c_int),
        ("tpc", ctypes.c_int * 4),
        ("n_k0", ctypes.c_int),
        ("k0", ctypes.c_int * 8),
        ("n_kmax", ctypes.c_int),
        ("kmax_mult", ctypes.c_int * 4),
        ("n_rho", ctypes.c_int),
        ("rho", ctypes.c_float * 8),
        ("reps", ctypes.c_int),
    ]


class VtTuneTrial(ctypes.Structure):
    _fields_ = [
        ("threads_per_cell", ctypes.c_int),
        ("k0", ctypes.c_int),
        ("k_max", ctypes.c_int),
        ("cls", ctypes.c_int),
        ("grid_density", ctypes.c_float),
        ("status", ctypes.c_int),
        ("ms", ctypes.c_double),
    ]


class VtTuneResult(ctypes.Structure):
    _fields_ = [
        ("best", VtParams),
        ("density_of_class", ctypes.c_float * VT_TUNE_CLASSES),
        ("best_ms", ctypes.c_double),
        ("n_tried", ctypes.c_int),
        ("tried", VtTuneTrial * VT_TUNE_MAX_TRIED),
    ]


class VtStats(ctypes.Structure):
    _fields_ = [
        ("passes", ctypes.c_int),
        ("k_of_pass", ctypes.c_int * VT_MAX_PASSES),
        ("cells_of_pass", ctypes.c_int64 * VT_MAX_PASSES),
        ("exhaustive_cells", ctypes.c_int64),
        ("capacity_retries", ctypes.c_int64),
        ("precision_retries", ctypes.c_int64),
        ("fp64_rechecks", ctypes.c_int64),
        ("unvalidated", ctypes.c_int64),
        ("grid_res", ctypes.c_int),
        ("launches", ctypes.c_int),
        ("clip_launches", ctypes.c_int),
        ("knn_launches", ctypes.c_int),
        ("ms_grid", ctypes.c_double),
        ("ms_knn", ctypes.c_double),
        ("ms_clip", ctypes.c_double),
        ("ms_emit", ctypes.c_double),
        ("ms_clip_pass", ctypes.c_double * VT_MAX_PASSES),
        ("clip_events", ctypes.c_int64 * 5),
        ("ms_knn_lists", ctypes.c_double),
        ("knn_candidates", ctypes.c_int64),
        ("knn_queries", ctypes.c_int64),
        ("walk_cells", ctypes.c_int64),
        ("walk_candidates", ctypes.c_int64),
    ]

    def as_dict(self) -> dict:
        p = self.passes
        m = min(p, VT_MAX_PASSES)
        return {
            "passes": p,
            "k_of_pass": list(self.k_of_pass[:m]),
            "cells_of_pass": list(self.cells_of_pass[:m]),
            "exhaustive_cells": self.exhaustive_cells,
            "capacity_retries": self.capacity_retries,
            "precision_retries": self.precision_retries,
            "fp64_rechecks": self.fp64_rechecks,
            "unvalidated": self.unvalidated,
            "grid_res": self.grid_res,
            "launches": self.launches,
            "clip_launches": self.clip_launches,
            "knn_launches": self.knn_launches,
            "ms_grid": self.ms_grid,
            "ms_knn": self.ms_knn,
            "ms_clip": self.ms_clip,
            "ms_emit": self.ms_emit,
            "ms_clip_pass": list(self.ms_clip_pass[:m]),
            "clip_events": list(self.clip_events),
            "ms_knn_lists": self.ms_knn_lists,
            "knn_candidates": self.knn_candidates,
            "knn_queries": self.knn_queries,
            "walk_cells": self.walk_cells,
            "walk_candidates": self.walk_candidates,
        }


class VtError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _build.LIB


def load() -> ctypes.CDLL:
    """Load libvt.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build()
        L = ctypes.CDLL(path)
        P, I64, I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        pp = ctypes.POINTER(VtParams)
        po = ctypes.POINTER(VtCellsOut)
        L.vt_params_default.argtypes = [pp]
        L.vt_params_default.restype = None
        L.vt_grid_resolution.argtypes = [pp, I64]
        L.vt_grid_resolution.restype = I
        L.vt_workspace_size.argtypes = [pp, I64, ctypes.POINTER(ctypes.c_size_t)]
        L.vt_workspace_size.restype = I
        L.vt_grid_build.argtypes = [P, I64, pp, I, P, P, P, P, ctypes.c_size_t, P]
        L.vt_grid_build.restype = I
        L.vt_knn.argtypes = [P, P, I, I64, P, I64, I, pp, P, P, P, ctypes.c_size_t, P]
        L.vt_knn.restype = I
        L.vt_clip_cells.argtypes = [P, P, I, I64, P, I64, P, P, I, pp, po, P, P, P, ctypes.c_size_t, P]
        L.vt_clip_cells.restype = I
        L.vt_emit.argtypes = [I64, pp, po, P, ctypes.c_size_t, P]
        L.vt_emit.restype = I
        L.vt_tessellate.argtypes = [P, I64, pp, po, ctypes.POINTER(VtStats), P, ctypes.c_size_t, P]
        L.vt_tessellate.restype = I
        L.vt_read_status.argtypes = [P, ctypes.c_size_t, P]
        L.vt_read_status.restype = I
        L.vt_last_error.argtypes = []
        L.vt_last_error.restype = ctypes.c_char_p
        L.vt_launch_count.argtypes = []
        L.vt_launch_count.restype = I64
        L.vt_version.argtypes = []
        L.vt_version.restype = ctypes.c_char_p
        L.vt_grid_build_static.argtypes = [P, I64, pp, I, P, P, P, P]
        L.vt_grid_build_static.restype = I
        L.vt_moments_adjoint.argtypes = [P, I64, po, P, P, P, pp, P, P]
        L.vt_moments_adjoint.restype = I
        L.vt_probe_fma.argtypes = [I, ctypes.POINTER(ctypes.c_double), P]
        L.vt_probe_fma.restype = I
        ps = ctypes.POINTER(VtStats)
        L.vt_batch_plan.argtypes = [P, I, pp, P, P, ctypes.POINTER(I64)]
        L.vt_batch_plan.restype = I
        L.vt_batch_workspace_size.argtypes = [pp, I64, I64, ctypes.POINTER(ctypes.c_size_t)]
        L.vt_batch_workspace_size.restype = I
        L.vt_tessellate_batch.argtypes = [P, I64, P, P, I, I64, pp, po, ps, P, ctypes.c_size_t, P]
        L.vt_tessellate_batch.restype = I
        L.vt_read_stats.argtypes = [P, ctypes.c_size_t, ps, po, P]
        L.vt_read_stats.restype = I
        L.vt_unvalidated_cells.argtypes = [pp, I64, P, I64, ctypes.POINTER(I64), P, ctypes.c_size_t, P]
        L.vt_unvalidated_cells.restype = I
        L.vt_lloyd_step.argtypes = [P, I64, P, P, pp, P, P]
        L.vt_lloyd_step.restype = I
        pts_ = ctypes.POINTER(VtTuneSpace)
        ptr_ = ctypes.POINTER(VtTuneResult)
        L.vt_cluster_index.argtypes = [P, I64, P, P, I, I64, pp, P, P, ctypes.c_size_t, P]
        L.vt_cluster_index.restype = I
        L.vt_cluster_class.argtypes = [ctypes.c_double]
        L.vt_cluster_class.restype = I
        L.vt_tune_space_default.argtypes = [pts_]
        L.vt_tune_space_default.restype = None
        L.vt_autotune_workspace_size.argtypes = [pp, pts_, I64, ctypes.POINTER(ctypes.c_size_t)]
        L.vt_autotune_workspace_size.restype = I
        L.vt_autotune.argtypes = [P, I64, pp, pts_, po, ptr_, P, ctypes.c_size_t, P]
        L.vt_autotune.restype = I
        L.vt_autotune_batch_workspace_size.argtypes = [P, I, pp, pts_, ctypes.POINTER(ctypes.c_size_t)]
        L.vt_autotune_batch_workspace_size.restype = I
        L.vt_autotune_batch.argtypes = [P, P, P, I, P, pp, pts_, P, po, ptr_, P, ctypes.c_size_t, P]
        L.vt_autotune_batch.restype = I
        _lib = L
        return L


def check(code: int) -> None:
    if code != VT_OK:
        raise VtError(code, load().vt_last_error().decode(errors="replace"))
