"""Seeded synthetic volumetric scenes and an instrumented path tracer.

This module is the input generator shared by the FP64 oracle (``oracle/``) and
the CUDA library. It holds no path-graph arithmetic: it traces paths and
records, per scattering vertex, what the paper's instrumented path tracer
records (Section 4): position, the outgoing direction, the phase-sampled
direction, the emitter sample and its pdf, the radiance found by the
phase-sampled direction and its emitter pdf, the medium coefficients, the
propagation weight tau/p_t of the segment entering the vertex, the successor
on the path, and the path tracer's own estimate of incoming indirect radiance.

The C core (``pgrec.c``) is compiled with gcc by :func:`build_lib`.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field, replace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libpgrec.so")
_lib = None


def build_lib(force: bool = False) -> str:
    """Compile the recorder with gcc (OpenMP when available)."""
    src = os.path.join(_HERE, "pgrec.c")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src)):
        return _LIB_PATH
    base = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", src, "-o", _LIB_PATH + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


class _Config(ctypes.Structure):
    _fields_ = [
        ("grid_res", ctypes.c_int32), ("medium_kind", ctypes.c_int32),
        ("sigma_t_max", ctypes.c_float), ("albedo", ctypes.c_float), ("g", ctypes.c_float),
        ("fbm_octaves", ctypes.c_int32), ("fbm_base_freq", ctypes.c_float),
        ("fbm_lacunarity", ctypes.c_float), ("fbm_gain", ctypes.c_float),
        ("cloud_threshold", ctypes.c_float), ("cloud_radius", ctypes.c_float),
        ("seed", ctypes.c_uint64),
        ("sun_dir", ctypes.c_float * 3), ("sun_irradiance", ctypes.c_float),
        ("sky_radiance", ctypes.c_float), ("area_radiance", ctypes.c_float),
        ("area_center", ctypes.c_float * 3), ("area_u", ctypes.c_float * 3),
        ("area_v", ctypes.c_float * 3), ("p_sun", ctypes.c_float), ("p_area", ctypes.c_float),
        ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("spp", ctypes.c_int32),
        ("max_depth", ctypes.c_int32),
        ("cam_pos", ctypes.c_float * 3), ("cam_target", ctypes.c_float * 3),
        ("cam_fov_deg", ctypes.c_float), ("extra_direct", ctypes.c_int32),
    ]


def _load():
    global _lib
    if _lib is None:
        build_lib()
        lib = ctypes.CDLL(_LIB_PATH)
        lib.pgrec_trace.restype = ctypes.c_void_p
        lib.pgrec_trace.argtypes = [ctypes.POINTER(_Config), ctypes.c_void_p, ctypes.c_int32]
        lib.pgrec_num_vertices.restype = ctypes.c_int64
        lib.pgrec_num_vertices.argtypes = [ctypes.c_void_p]
        lib.pgrec_num_paths.restype = ctypes.c_int64
        lib.pgrec_num_paths.argtypes = [ctypes.c_void_p]
        lib.pgrec_majorant.restype = ctypes.c_double
        lib.pgrec_majorant.argtypes = [ctypes.c_void_p]
        lib.pgrec_copy_vertices.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)] + [ctypes.c_void_p] * 4
        lib.pgrec_copy_paths.argtypes = [ctypes.c_void_p] * 4
        lib.pgrec_copy_medium.argtypes = [ctypes.c_void_p] * 3
        lib.pgrec_copy_extra.argtypes = [ctypes.c_void_p] * 7
        lib.pgrec_build_medium.argtypes = [ctypes.POINTER(_Config), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.pgrec_log.argtypes = [ctypes.c_float]
        lib.pgrec_log.restype = ctypes.c_float
        lib.pgrec_sincos_2pi.argtypes = [ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p]
        lib.pgrec_free.argtypes = [ctypes.c_void_p]
        _lib = lib
    return _lib


def medium(scene: "Scene", albedo_grid: np.ndarray | None = None) -> tuple:
    """The scene's (density, albedo) voxel grids, float32, grid_res^3 each
    (index x + G (y + G z)), as :func:`trace` builds them."""
    lib = _load()
    G = scene.grid_res
    dens = np.empty(G ** 3, np.float32)
    alb = np.empty(G ** 3, np.float32)
    ag = None
    if albedo_grid is not None:
        ag = np.ascontiguousarray(albedo_grid, dtype=np.float32)
    cfg = scene._cstruct()
    lib.pgrec_build_medium(ctypes.byref(cfg), ag.ctypes.data if ag is not None else None, dens.ctypes.data,
                           alb.ctypes.data)
    return dens, alb


def elementary(name: str, x: float):
    """The recorder's own single-precision log (``"log"``) or (sin, cos) of
    2 pi x (``"sincos_2pi"``), x rounded to float32 first."""
    lib = _load()
    if name == "log":
        return lib.pgrec_log(x)
    s, c = ctypes.c_float(), ctypes.c_float()
    lib.pgrec_sincos_2pi(x, ctypes.byref(s), ctypes.byref(c))
    return s.value, c.value


@dataclass(frozen=True)
class Scene:
    """One synthetic workload: medium, lights, camera and path-graph settings."""
    name: str
    grid_res: int
    medium_kind: int            # 0 constant, 1 fBm cloud
    sigma_t_max: float
    albedo: float
    g: float
    width: int
    height: int
    spp: int
    max_depth: int
    k: int                      # neighbours per row, self included
    iters: int                  # propagation sweeps
    seed: int = 0
    fbm_octaves: int = 5
    fbm_base_freq: float = 4.0
    fbm_lacunarity: float = 2.0
    fbm_gain: float = 0.5
    cloud_threshold: float = 0.15
    cloud_radius: float = 0.7
    sun_dir: tuple = (-0.35, -1.0, 0.25)
    sun_irradiance: float = 0.0
    sky_radiance: float = 0.0
    area_radiance: float = 0.0
    area_center: tuple = (0.5, 1.6, 0.5)
    area_u: tuple = (0.0, 0.0, 0.3)
    area_v: tuple = (0.3, 0.0, 0.0)
    p_sun: float = 0.5
    p_area: float = 0.5
    cam_pos: tuple = (0.5, 0.5, -1.6)
    cam_target: tuple = (0.5, 0.5, 0.5)
    cam_fov_deg: float = 26.0
    extra_direct: int = 0       # extra emitter samples per path at its first vertex
    weight_dtypes: tuple = ("f32",)
    extra: dict = field(default_factory=dict)

    def with_(self, **kw) -> "Scene":
        return replace(self, **kw)

    def _cstruct(self) -> _Config:
        c = _Config()
        for f, _ in _Config._fields_:
            v = getattr(self, f)
            if isinstance(v, tuple):
                arr = getattr(c, f)
                for i, x in enumerate(v):
                    arr[i] = x
            else:
                setattr(c, f, v)
        return c


# The five workloads. Media are synthetic stand-ins for the paper's scenes
# (clouds and smoke under sun/sky or area lighting).
CUBE_CONST = Scene(
    name="cube32_const_sigma2_a0.9_iso_64px_4spp_d8", grid_res=32, medium_kind=0,
    sigma_t_max=2.0, albedo=0.9, g=0.0, width=64, height=64, spp=4, max_depth=8,
    k=8, iters=10, sun_irradiance=1.0, sun_dir=(-0.35, -1.0, 0.25), cam_fov_deg=24.0)
CLOUD128 = Scene(
    name="cloud128_fbm_sigma20_a0.99_g0.8_256px_16spp_d64", grid_res=128, medium_kind=1,
    sigma_t_max=20.0, albedo=0.99, g=0.8, width=256, height=256, spp=16, max_depth=64,
    k=16, iters=30, sun_irradiance=2.0, sky_radiance=0.3, p_sun=0.5)
CLOUD128_16BIT = CLOUD128.with_(weight_dtypes=("f32", "u16", "f16", "bf16"))
CLOUD64_GRAD = Scene(
    name="cloud64_fbm_a0.95_g0.6_128px_8spp_d32", grid_res=64, medium_kind=1,
    sigma_t_max=20.0, albedo=0.95, g=0.6, width=128, height=128, spp=8, max_depth=32,
    k=16, iters=20, sun_irradiance=2.0, sky_radiance=0.3, p_sun=0.5)
CLOUD256_DENSE = Scene(
    name="cloud256_fbm_sigma60_a0.999_g0.9_1024px_8spp_d256", grid_res=256, medium_kind=1,
    sigma_t_max=60.0, albedo=0.999, g=0.9, width=1024, height=1024, spp=8, max_depth=256,
    k=16, iters=50, area_radiance=5.0, sky_radiance=0.2, p_area=0.5, cloud_threshold=0.2,
    weight_dtypes=("u16",))

SCENES = {s.name: s for s in (CUBE_CONST, CLOUD128, CLOUD64_GRAD, CLOUD256_DENSE)}

EXTRA_F32 = ("x_ex", "x_ey", "x_ez", "x_Le", "x_pe")
F32_FIELDS = ("px", "py", "pz", "ox", "oy", "oz", "dx", "dy", "dz", "ex", "ey", "ez",
              "g", "sigma_s", "sigma_t", "w_prop", "Le", "pe_e", "Lph", "pe_ph", "L0")


def trace(scene: Scene, nthreads: int = 0, albedo_grid: np.ndarray | None = None,
          alloc=None) -> dict:
    """Trace ``scene`` and return its records as a dict of numpy arrays.

    ``alloc(shape, dtype)`` may supply the output buffers (e.g. pinned host
    tensors viewed as numpy); the default is ``np.empty``.
    With ``scene.extra_direct`` = M > 0 also the extra emitter samples drawn
    at each path's first vertex: ``x_ex, x_ey, x_ez, x_Le, x_pe`` (float32)
    and ``x_delta`` (uint8), M per path, path p's at [p*M, (p+1)*M) (paths
    without a vertex hold Le = 0).
    Keys: the per-vertex float32 fields in ``F32_FIELDS``, ``L0_f64``,
    ``e_delta`` (uint8), ``succ`` and ``voxel`` (int32); per path ``first``
    (int32), ``bg`` (float32) and ``pt_value`` (float64); the medium
    ``density`` and ``albedo_grid``; ``pt_image`` (float64, the path tracer's
    own image) and scalars ``n``, ``n_paths``, ``majorant``.
    """
    lib = _load()
    alloc = alloc or (lambda shape, dtype: np.empty(shape, dtype))
    cfg = scene._cstruct()
    ag = None
    if albedo_grid is not None:
        ag = np.ascontiguousarray(albedo_grid, dtype=np.float32)
        assert ag.size == scene.grid_res ** 3
    h = lib.pgrec_trace(ctypes.byref(cfg), ag.ctypes.data if ag is not None else None, nthreads)
    try:
        n = lib.pgrec_num_vertices(h)
        P = lib.pgrec_num_paths(h)
        out = {f: alloc((n,), np.float32) for f in F32_FIELDS}
        out["L0_f64"] = alloc((n,), np.float64)
        out["e_delta"] = alloc((n,), np.uint8)
        out["succ"] = alloc((n,), np.int32)
        out["voxel"] = alloc((n,), np.int32)
        ptrs = (ctypes.c_void_p * len(F32_FIELDS))(*[out[f].ctypes.data for f in F32_FIELDS])
        lib.pgrec_copy_vertices(h, ptrs, out["L0_f64"].ctypes.data, out["e_delta"].ctypes.data,
                                out["succ"].ctypes.data, out["voxel"].ctypes.data)
        out["first"] = alloc((P,), np.int32)
        out["bg"] = alloc((P,), np.float32)
        out["pt_value"] = np.empty(P, np.float64)
        lib.pgrec_copy_paths(h, out["first"].ctypes.data, out["bg"].ctypes.data, out["pt_value"].ctypes.data)
        G = scene.grid_res
        out["density"] = np.empty(G ** 3, np.float32)
        out["albedo_grid"] = np.empty(G ** 3, np.float32)
        lib.pgrec_copy_medium(h, out["density"].ctypes.data, out["albedo_grid"].ctypes.data)
        out["majorant"] = lib.pgrec_majorant(h)
        M = int(scene.extra_direct)
        if M > 0:
            for f in EXTRA_F32:
                out[f] = alloc((P * M,), np.float32)
            out["x_delta"] = alloc((P * M,), np.uint8)
            lib.pgrec_copy_extra(h, *[out[f].ctypes.data for f in EXTRA_F32], out["x_delta"].ctypes.data)
        out["extra_direct"] = M
    finally:
        lib.pgrec_free(h)
    out["n"] = int(n)
    out["n_paths"] = int(P)
    out["pt_image"] = out["pt_value"].reshape(scene.height, scene.width, scene.spp).mean(axis=2)
    out["spp"] = scene.spp
    out["width"] = scene.width
    out["height"] = scene.height
    return out


def _copy_extra(rec: dict, out: dict, paths) -> None:
    """Extra first-vertex samples of the chosen paths, in their new order."""
    M = int(rec.get("extra_direct", 0))
    out["extra_direct"] = M
    if M == 0:
        return
    q = (np.asarray(paths, np.int64)[:, None] * M + np.arange(M)[None, :]).reshape(-1)
    for f in EXTRA_F32 + ("x_delta",):
        out[f] = np.ascontiguousarray(rec[f][q])


def subset_paths(rec: dict, path_lo: int, path_hi: int) -> dict:
    """Records of paths [path_lo, path_hi) only, re-indexed from zero.

    Paths are contiguous in the vertex array, so the subset is a slice.
    """
    first = rec["first"][path_lo:path_hi]
    vs = first[first >= 0]
    if vs.size == 0:
        v0 = v1 = 0
    else:
        v0 = int(vs.min())
        # last vertex of the last non-empty path: walk its successor chain
        v = int(vs.max())
        while rec["succ"][v] >= 0:
            v = int(rec["succ"][v])
        v1 = v + 1
    out = {}
    for f in F32_FIELDS + ("L0_f64", "e_delta", "voxel"):
        out[f] = np.ascontiguousarray(rec[f][v0:v1])
    succ = rec["succ"][v0:v1].astype(np.int64)
    out["succ"] = np.where(succ >= 0, succ - v0, -1).astype(np.int32)
    out["first"] = np.where(first >= 0, first - v0, -1).astype(np.int32)
    out["bg"] = np.ascontiguousarray(rec["bg"][path_lo:path_hi])
    out["pt_value"] = np.ascontiguousarray(rec["pt_value"][path_lo:path_hi])
    _copy_extra(rec, out, np.arange(path_lo, path_hi))
    for k in ("density", "albedo_grid", "majorant", "spp"):
        out[k] = rec[k]
    out["n"] = v1 - v0
    out["n_paths"] = path_hi - path_lo
    return out


def sample_pixels(rec: dict, width: int, height: int, spp: int, stride: int, offset=(0, 0)) -> dict:
    """Records of the paths of every `stride`-th pixel in x and y (all spp),
    starting at pixel ``offset`` = (y, x), re-indexed from zero; the result is
    a (height/stride x width/stride) image's worth of paths with every path's
    vertices still contiguous."""
    ys = np.arange(offset[0], height, stride)
    xs = np.arange(offset[1], width, stride)
    pix = (ys[:, None] * width + xs[None, :]).reshape(-1)
    paths = (pix[:, None] * spp + np.arange(spp)[None, :]).reshape(-1)
    first = rec["first"][paths]
    # vertex ranges of the chosen paths (a path runs from first along succ)
    starts, lens = [], []
    succ = rec["succ"]
    for f in first:
        if f < 0:
            lens.append(0)
            starts.append(0)
            continue
        v, ln = int(f), 1
        while succ[v] >= 0:
            v = int(succ[v])
            ln += 1
        starts.append(int(f))
        lens.append(ln)
    lens = np.array(lens, np.int64)
    starts = np.array(starts, np.int64)
    idx = np.concatenate([np.arange(s, s + ln) for s, ln in zip(starts, lens) if ln > 0]) if lens.sum() else \
        np.zeros(0, np.int64)
    new_first = np.where(lens > 0, np.concatenate([[0], np.cumsum(lens)[:-1]]), -1).astype(np.int32)
    out = {f: np.ascontiguousarray(rec[f][idx]) for f in F32_FIELDS + ("L0_f64", "e_delta", "voxel")}
    old2new = np.full(rec["n"], -1, np.int64)
    old2new[idx] = np.arange(len(idx))
    s = succ[idx].astype(np.int64)
    out["succ"] = np.where(s >= 0, old2new[np.where(s >= 0, s, 0)], -1).astype(np.int32)
    out["first"] = new_first
    out["bg"] = np.ascontiguousarray(rec["bg"][paths])
    out["pt_value"] = np.ascontiguousarray(rec["pt_value"][paths])
    _copy_extra(rec, out, paths)
    for k in ("density", "albedo_grid", "majorant"):
        out[k] = rec[k]
    out["spp"] = spp
    out["width"] = len(xs)
    out["height"] = len(ys)
    out["n"] = int(len(idx))
    out["n_paths"] = int(len(paths))
    return out
