"""ctypes declarations of the libpg C ABI (include/pg.h)."""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpg.so")

PG_STATUS = {
    0: "ok", 1: "invalid argument", 2: "out of device memory", 3: "CUDA error",
    4: "non-finite input", 5: "device wait timed out", 6: "unsupported parameter", 7: "invalid call order",
}
W_DTYPES = {"f32": 0, "bf16": 1, "f16": 2, "u16": 3}

c_float_p = ctypes.POINTER(ctypes.c_float)


class PgVertices(ctypes.Structure):
    _fields_ = [(name, ctypes.c_void_p) for name in (
        "px", "py", "pz", "ox", "oy", "oz", "dx", "dy", "dz", "ex", "ey", "ez",
        "g", "sigma_s", "sigma_t", "w_prop", "Le", "pe_e", "Lph", "pe_ph", "e_delta", "succ")]


class PgBuildParams(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("bbox_lo", ctypes.c_float * 3), ("bbox_hi", ctypes.c_float * 3),
                ("r2_max", ctypes.c_int64), ("grid_level", ctypes.c_int32), ("cluster_size", ctypes.c_int32),
                ("cluster_seed", ctypes.c_uint64)]


class PgGraphInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("k", ctypes.c_int32), ("row_width", ctypes.c_int32),
                ("grid_level", ctypes.c_int32), ("aggregated", ctypes.c_int32), ("n_active", ctypes.c_int64),
                ("nnz_swept", ctypes.c_int64), ("device_bytes", ctypes.c_int64), ("weight_dtype", ctypes.c_int32),
                ("history_iters", ctypes.c_int32), ("knn_exact", ctypes.c_int64), ("clusters", ctypes.c_int64)]


class PgExtraSamples(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32)] + [(name, ctypes.c_void_p) for name in ("ex", "ey", "ez", "Le", "pe_e", "e_delta")]


class PgOutputParams(ctypes.Structure):
    _fields_ = [("final_gather_k", ctypes.c_int32), ("extra", ctypes.POINTER(PgExtraSamples)),
                ("fg_nbr", ctypes.c_void_p)]


class PgScene(ctypes.Structure):
    _fields_ = [("grid_res", ctypes.c_int32), ("density", ctypes.c_void_p), ("albedo", ctypes.c_void_p),
                ("g", ctypes.c_float), ("sun_dir", ctypes.c_float * 3), ("sun_irradiance", ctypes.c_float),
                ("sky_radiance", ctypes.c_float), ("area_radiance", ctypes.c_float),
                ("area_center", ctypes.c_float * 3), ("area_u", ctypes.c_float * 3), ("area_v", ctypes.c_float * 3),
                ("p_sun", ctypes.c_float), ("p_area", ctypes.c_float), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32), ("spp", ctypes.c_int32), ("max_depth", ctypes.c_int32),
                ("cam_pos", ctypes.c_float * 3), ("cam_target", ctypes.c_float * 3), ("cam_fov_deg", ctypes.c_float),
                ("seed", ctypes.c_uint64), ("extra_direct", ctypes.c_int32)]


RECORD_VERTEX_F32 = ("px", "py", "pz", "ox", "oy", "oz", "dx", "dy", "dz", "ex", "ey", "ez", "g", "sigma_s",
                     "sigma_t", "w_prop", "Le", "pe_e", "Lph", "pe_ph", "L0")
RECORD_EXTRA_F32 = ("x_ex", "x_ey", "x_ez", "x_Le", "x_pe")


class PgRecording(ctypes.Structure):
    _fields_ = ([(k, ctypes.c_void_p) for k in RECORD_VERTEX_F32]
                + [(k, ctypes.c_void_p) for k in ("L0_f64", "e_delta", "succ", "voxel", "first", "bg", "val")]
                + [(k, ctypes.c_void_p) for k in RECORD_EXTRA_F32 + ("x_delta",)])


class PgShardInfo(ctypes.Structure):
    _fields_ = [("n_shards", ctypes.c_int32), ("shard", ctypes.c_int32), ("row_width", ctypes.c_int32),
                ("row_begin", ctypes.c_int64), ("row_end", ctypes.c_int64), ("n_halo", ctypes.c_int64),
                ("local_len", ctypes.c_int64), ("n_send", ctypes.c_int64)]


class PgStepParams(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("iters", ctypes.c_int32), ("wdtype", ctypes.c_int),
                ("bbox_lo", ctypes.c_float * 3), ("bbox_hi", ctypes.c_float * 3), ("spp", ctypes.c_int32),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("adjoint", ctypes.c_int32),
                ("n_vox", ctypes.c_int64)]


EXPORTS = ("pg_build_graph", "pg_graph_neighbors", "pg_graph_get_info", "pg_aggregate", "pg_propagate",
           "pg_gather", "pg_propagate_adjoint", "pg_graph_release_weights", "pg_graph_destroy",
           "pg_status_string", "pg_launch_count", "pg_propagate_noalloc", "pg_gather_ex",
           "pg_record_count", "pg_record_fill", "pg_prepare_adjoint", "pg_shard_create", "pg_shard_create_host",
           "pg_shard_get_info", "pg_shard_get_lists", "pg_shard_load", "pg_shard_pack", "pg_shard_sweep",
           "pg_shard_destroy", "pg_graph_y_from_L", "pg_graph_L_from_y", "pg_step_host")

_lib = None


def load(path: str = LIB_PATH):
    """Load libpg.so; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libpg.so not found at {path}: run paper_2404_11894_gb300.build.build() first")
    lib = ctypes.CDLL(path)
    vp, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    lib.pg_build_graph.argtypes = [ctypes.POINTER(PgVertices), i64, ctypes.POINTER(PgBuildParams), vp,
                                   ctypes.POINTER(vp)]
    lib.pg_graph_neighbors.argtypes = [vp, vp, vp]
    lib.pg_graph_get_info.argtypes = [vp, ctypes.POINTER(PgGraphInfo)]
    lib.pg_aggregate.argtypes = [vp, ctypes.POINTER(PgVertices), ctypes.c_int, vp, vp, vp]
    lib.pg_propagate.argtypes = [vp, vp, vp, i32, f64, i32, vp, vp, vp, vp]
    lib.pg_gather.argtypes = [vp, vp, vp, vp, vp, i64, i32, i32, i32, vp, vp]
    lib.pg_record_count.argtypes = [ctypes.POINTER(PgScene), vp, ctypes.POINTER(i64), vp]
    lib.pg_record_fill.argtypes = [ctypes.POINTER(PgScene), vp, ctypes.POINTER(PgRecording), vp]
    lib.pg_gather_ex.argtypes = [vp, vp, vp, vp, vp, i64, i32, i32, i32, ctypes.POINTER(PgOutputParams), vp, vp]
    lib.pg_propagate_adjoint.argtypes = [vp, vp, vp, i64, i32, i32, i32, vp, vp, vp, vp, vp, i64, i32, vp]
    lib.pg_graph_release_weights.argtypes = [vp]
    lib.pg_prepare_adjoint.argtypes = [vp, vp]
    lib.pg_graph_destroy.argtypes = [vp]
    lib.pg_graph_destroy.restype = None
    lib.pg_status_string.argtypes = [ctypes.c_int]
    lib.pg_status_string.restype = ctypes.c_char_p
    lib.pg_propagate_noalloc.argtypes = [vp, vp, i32, f64, vp, vp]
    lib.pg_shard_create.argtypes = [vp, i32, i32, vp, ctypes.POINTER(vp)]
    lib.pg_shard_create_host.argtypes = [vp, i64, i32, i64, i32, i32, ctypes.POINTER(vp)]
    lib.pg_shard_get_info.argtypes = [vp, ctypes.POINTER(PgShardInfo)]
    lib.pg_shard_get_lists.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    lib.pg_shard_load.argtypes = [vp, vp, vp, vp]
    lib.pg_shard_pack.argtypes = [vp, vp, vp, vp]
    lib.pg_shard_sweep.argtypes = [vp, vp, vp, vp]
    lib.pg_shard_destroy.argtypes = [vp]
    lib.pg_shard_destroy.restype = None
    lib.pg_graph_y_from_L.argtypes = [vp, vp, vp, vp]
    lib.pg_graph_L_from_y.argtypes = [vp, vp, vp, vp]
    lib.pg_step_host.argtypes = [ctypes.POINTER(PgVertices), i64, vp, vp, vp, i64, vp, vp,
                                 ctypes.POINTER(PgStepParams), vp, vp, vp, vp]
    lib.pg_launch_count.argtypes = []
    lib.pg_launch_count.restype = ctypes.c_int64
    for name in EXPORTS:
        if name not in ("pg_graph_destroy", "pg_status_string", "pg_launch_count", "pg_shard_destroy"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


class PgError(RuntimeError):
    def __init__(self, status: int, call: str):
        self.status = status
        super().__init__(f"{call}: {PG_STATUS.get(status, status)} (status {status})")


def check(status: int, call: str):
    if status != 0:
        raise PgError(status, call)
