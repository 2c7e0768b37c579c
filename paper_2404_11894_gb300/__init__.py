"""GB300 volumetric path-graph hot path: Python binding of libpg (include/pg.h).

The functions below carry the C names and only marshal arguments: torch
tensors provide device memory and the current CUDA stream; every step of the
path runs in the library's CUDA kernels. There is no CPU fallback: importing
the binding fails when libpg.so has not been built.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import PgBuildParams, PgError, PgGraphInfo, PgVertices, W_DTYPES, check

VERTEX_F32 = ("px", "py", "pz", "ox", "oy", "oz", "dx", "dy", "dz", "ex", "ey", "ez",
              "g", "sigma_s", "sigma_t", "w_prop", "Le", "pe_e", "Lph", "pe_ph")

_LIB = _lib.load()


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "device tensors must be contiguous CUDA tensors"
    return ctypes.c_void_p(t.data_ptr())


class Vertices:
    """Per-vertex records on the device (caller order), see pg_vertices."""

    def __init__(self, tensors: dict):
        self.t = tensors
        self.n = int(tensors["px"].numel())
        self._struct = PgVertices(**{k: (tensors[k].data_ptr() if k in tensors else None)
                                     for k, _ in PgVertices._fields_})

    @staticmethod
    def from_records(rec: dict, device="cuda", non_blocking=False, overrides: dict | None = None) -> "Vertices":
        """Copy recorder output (numpy or host tensors) to the device."""
        t = {}
        for k in VERTEX_F32 + ("e_delta", "succ"):
            src = (overrides or {}).get(k, rec[k])
            if isinstance(src, np.ndarray):
                src = torch.from_numpy(np.ascontiguousarray(src))
            t[k] = src.to(device, non_blocking=non_blocking)
        return Vertices(t)

    @property
    def struct(self) -> PgVertices:
        return self._struct


class Graph:
    """Owns a pg_graph handle; destroyed with the object."""

    def __init__(self, handle: ctypes.c_void_p, n: int, k: int):
        self.handle = handle
        self.n = n
        self.k = k

    def info(self) -> dict:
        inf = PgGraphInfo()
        check(_LIB.pg_graph_get_info(self.handle, ctypes.byref(inf)), "pg_graph_get_info")
        return {f: getattr(inf, f) for f, _ in PgGraphInfo._fields_}

    def neighbors(self, stream=None) -> torch.Tensor:
        out = torch.empty((self.n, self.k), dtype=torch.int32, device="cuda")
        check(_LIB.pg_graph_neighbors(self.handle, _ptr(out), _stream_ptr(stream)), "pg_graph_neighbors")
        return out

    def release_weights(self):
        check(_LIB.pg_graph_release_weights(self.handle), "pg_graph_release_weights")

    def close(self):
        if self.handle:
            _LIB.pg_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pg_build_graph(verts: Vertices, k: int, bbox_lo=(0.0, 0.0, 0.0), bbox_hi=(1.0, 1.0, 1.0), r2_max: int = -1,
                   grid_level: int = 0, cluster_size: int = 0, cluster_seed: int = 0, stream=None) -> Graph:
    """kNN neighbourhoods, or with ``cluster_size`` K > 0 the paper's disjoint
    clusters of expected size K (parts of at most k points)."""
    p = PgBuildParams()
    p.k = k
    for a in range(3):
        p.bbox_lo[a] = bbox_lo[a]
        p.bbox_hi[a] = bbox_hi[a]
    p.r2_max = r2_max
    p.grid_level = grid_level
    p.cluster_size = cluster_size
    p.cluster_seed = cluster_seed
    h = ctypes.c_void_p()
    check(_LIB.pg_build_graph(ctypes.byref(verts.struct), verts.n, ctypes.byref(p), _stream_ptr(stream),
                              ctypes.byref(h)), "pg_build_graph")
    return Graph(h, verts.n, k)


def pg_aggregate(graph: Graph, verts: Vertices, wdtype: str = "f32", stream=None):
    """Returns (c, D), caller order, float32 device tensors."""
    c = torch.empty(graph.n, dtype=torch.float32, device="cuda")
    D = torch.empty(graph.n, dtype=torch.float32, device="cuda")
    check(_LIB.pg_aggregate(graph.handle, ctypes.byref(verts.struct), W_DTYPES[wdtype], _ptr(c), _ptr(D),
                            _stream_ptr(stream)), "pg_aggregate")
    return c, D


def pg_propagate(graph: Graph, L0: torch.Tensor, iters: int, c: torch.Tensor | None = None, tol: float = 0.0,
                 keep_history: bool = False, want_residual: bool = False, out: torch.Tensor | None = None,
                 stream=None):
    """Returns L (caller order); with want_residual also (residuals, iters_done)."""
    L = out if out is not None else torch.empty(graph.n, dtype=torch.float32, device="cuda")
    res = (ctypes.c_double * max(iters, 1))() if want_residual else None
    done = ctypes.c_int32(0) if want_residual else None
    check(_LIB.pg_propagate(graph.handle, _ptr(c), _ptr(L0), iters, tol, int(keep_history), _ptr(L),
                            res, ctypes.byref(done) if done is not None else None, _stream_ptr(stream)),
          "pg_propagate")
    if want_residual:
        return L, np.array(res[:iters]), done.value
    return L


def pg_gather(graph: Graph, L: torch.Tensor, D: torch.Tensor, first: torch.Tensor, bg: torch.Tensor, spp: int,
              width: int, height: int, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    img = out if out is not None else torch.empty((height, width), dtype=torch.float32, device="cuda")
    check(_LIB.pg_gather(graph.handle, _ptr(L), _ptr(D), _ptr(first), _ptr(bg), first.numel(), spp, width, height,
                         _ptr(img), _stream_ptr(stream)), "pg_gather")
    return img


EXTRA_FIELDS = ("ex", "ey", "ez", "Le", "pe_e", "e_delta")


def pg_gather_ex(graph: Graph, L: torch.Tensor, D: torch.Tensor | None, first: torch.Tensor, bg: torch.Tensor,
                 spp: int, width: int, height: int, final_gather_k: int = 0, extra: dict | None = None,
                 want_fg_nbr: bool = False, out: torch.Tensor | None = None, stream=None):
    """pg_gather with the output options of include/pg.h: a final gather over
    the ``final_gather_k`` nearest vertices of each first vertex, and/or the
    direct term from ``extra`` = {"m": M, "ex", "ey", "ez", "Le", "pe_e",
    "e_delta": device tensors of n_paths*M entries}. Returns the image, and
    with ``want_fg_nbr`` also the final gather's neighbour table."""
    img = out if out is not None else torch.empty((height, width), dtype=torch.float32, device="cuda")
    xs = None
    if extra is not None:
        xs = _lib.PgExtraSamples(m=int(extra["m"]), **{k: extra[k].data_ptr() for k in EXTRA_FIELDS})
        for k in EXTRA_FIELDS:
            _ptr(extra[k])
    fg = torch.empty((first.numel(), final_gather_k), dtype=torch.int32, device="cuda") \
        if want_fg_nbr and final_gather_k > 0 else None
    p = _lib.PgOutputParams(final_gather_k=final_gather_k, extra=ctypes.pointer(xs) if xs is not None else None,
                            fg_nbr=fg.data_ptr() if fg is not None else None)
    check(_LIB.pg_gather_ex(graph.handle, _ptr(L), _ptr(D), _ptr(first), _ptr(bg), first.numel(), spp, width,
                            height, ctypes.byref(p), _ptr(img), _stream_ptr(stream)), "pg_gather_ex")
    return (img, fg) if want_fg_nbr else img


def extra_from_records(rec: dict, device="cuda") -> dict:
    """The recorder's extra first-vertex samples (x_ex ... x_delta) as the
    device tensors pg_gather_ex takes."""
    names = {"ex": "x_ex", "ey": "x_ey", "ez": "x_ez", "Le": "x_Le", "pe_e": "x_pe", "e_delta": "x_delta"}
    out = {k: torch.from_numpy(np.ascontiguousarray(rec[v])).to(device) for k, v in names.items()}
    out["m"] = int(rec["extra_direct"])
    return out


SCENE_FIELDS = tuple(f for f, _ in _lib.PgScene._fields_ if f not in ("density", "albedo"))


def pg_step_host(host: dict, spp: int, width: int, height: int, k: int, iters: int, wdtype: str = "f32",
                 target=None, n_vox: int = 0, want_sigma_s: bool = False, bbox_lo=(0.0, 0.0, 0.0),
                 bbox_hi=(1.0, 1.0, 1.0), out: dict | None = None, stream=None) -> dict:
    """The whole hot path from HOST buffers through the C ABI (pg_step_host):
    ``host`` holds CPU tensors (pinned for overlapped copies) of the vertex
    records, ``L0``, ``first``, ``bg`` (and ``voxel`` with n_vox > 0); with a
    host ``target`` image the adjoint of the L2 loss runs too. Returns host
    tensors: image, and grad_sigma_s / grad_albedo when requested (written
    into ``out``'s tensors of those names when given: pinned buffers let the
    device-to-host copies run asynchronously)."""
    def hp(t):
        return ctypes.c_void_p(t.data_ptr()) if t is not None else None

    vs = PgVertices(**{k_: (host[k_].data_ptr() if k_ in host else None) for k_, _ in PgVertices._fields_})
    n = int(host["px"].numel())
    P = int(host["first"].numel())
    prm = _lib.PgStepParams(k=k, iters=iters, wdtype=W_DTYPES[wdtype], spp=spp, width=width, height=height,
                            adjoint=1 if target is not None else 0, n_vox=n_vox)
    for i in range(3):
        prm.bbox_lo[i], prm.bbox_hi[i] = bbox_lo[i], bbox_hi[i]
    out = out or {}

    def buf(name, shape, want):
        if not want:
            return None
        t = out.get(name)
        if t is None or tuple(t.shape) != tuple(shape):
            t = torch.empty(shape, dtype=torch.float32)
        return t

    img = buf("image", (height, width), True)
    gs = buf("grad_sigma_s", (n,), want_sigma_s and target is not None)
    ga = buf("grad_albedo", (n_vox,), n_vox > 0 and target is not None)
    check(_LIB.pg_step_host(ctypes.byref(vs), n, hp(host["L0"]), hp(host["first"]), hp(host["bg"]), P, hp(target),
                            hp(host.get("voxel")) if ga is not None else None, ctypes.byref(prm), hp(img), hp(gs),
                            hp(ga), _stream_ptr(stream)), "pg_step_host")
    return {"image": img, "grad_sigma_s": gs, "grad_albedo": ga}


def pg_record(scene, density: torch.Tensor, albedo: torch.Tensor, stream=None) -> dict:
    """The GPU path recorder (pg_record_count + pg_record_fill). ``scene``:
    any object (or dict) carrying the pg_scene fields by name; ``density``,
    ``albedo``: device float32 grids of grid_res^3 voxels. Returns device
    tensors keyed like the host recorder's output: the per-vertex fields,
    ``L0_f64``, ``e_delta``, ``succ``, ``voxel``; per path ``first``, ``bg``,
    ``pt_value``; the extra first-vertex samples ``x_*`` when requested; and
    ``n``, ``n_paths``, ``extra_direct``."""
    get = (lambda k: scene[k]) if isinstance(scene, dict) else (lambda k: getattr(scene, k))  # noqa: E731
    sc = _lib.PgScene()
    for f in SCENE_FIELDS:
        v = get(f)
        if isinstance(v, (tuple, list)):
            arr = getattr(sc, f)
            for i, x in enumerate(v):
                arr[i] = x
        else:
            setattr(sc, f, v)
    sc.density, sc.albedo = _ptr(density).value, _ptr(albedo).value
    P = int(sc.width) * int(sc.height) * int(sc.spp)
    offsets = torch.empty(P + 1, dtype=torch.int64, device="cuda")
    n = ctypes.c_int64(0)
    check(_LIB.pg_record_count(ctypes.byref(sc), _ptr(offsets), ctypes.byref(n), _stream_ptr(stream)),
          "pg_record_count")
    n = int(n.value)
    M = int(sc.extra_direct)
    dev = torch.device("cuda")
    nb = max(n, 1)  # never a NULL vertex array, even when no ray hits the medium
    out = {k: torch.empty(nb, dtype=torch.float32, device=dev) for k in _lib.RECORD_VERTEX_F32}
    out["L0_f64"] = torch.empty(nb, dtype=torch.float64, device=dev)
    out["e_delta"] = torch.empty(nb, dtype=torch.uint8, device=dev)
    out["succ"] = torch.empty(nb, dtype=torch.int32, device=dev)
    out["voxel"] = torch.empty(nb, dtype=torch.int32, device=dev)
    out["first"] = torch.empty(P, dtype=torch.int32, device=dev)
    out["bg"] = torch.empty(P, dtype=torch.float32, device=dev)
    out["pt_value"] = torch.empty(P, dtype=torch.float64, device=dev)
    if M > 0:
        for k in _lib.RECORD_EXTRA_F32:
            out[k] = torch.empty(P * M, dtype=torch.float32, device=dev)
        out["x_delta"] = torch.empty(P * M, dtype=torch.uint8, device=dev)
    rec = _lib.PgRecording(**{k: out[k].data_ptr() for k in out if k != "pt_value"}, val=out["pt_value"].data_ptr())
    check(_LIB.pg_record_fill(ctypes.byref(sc), _ptr(offsets), ctypes.byref(rec), _stream_ptr(stream)),
          "pg_record_fill")
    if n == 0:
        for k in list(_lib.RECORD_VERTEX_F32) + ["L0_f64", "e_delta", "succ", "voxel"]:
            out[k] = out[k][:0]
    out["n"], out["n_paths"], out["extra_direct"] = n, P, M
    return out


def pg_propagate_adjoint(graph: Graph, dI: torch.Tensor, first: torch.Tensor, spp: int, width: int, height: int,
                         want_sigma_s: bool = True, want_g: bool = True, voxel: torch.Tensor | None = None,
                         sigma_t: torch.Tensor | None = None, n_vox: int = 0, recompute_weights: int = 0,
                         stream=None) -> dict:
    """recompute_weights: 0 transposed copy (deterministic), 1 re-evaluate
    weights, 2 stored rows with atomic scatter (see include/pg.h)."""
    gs = torch.empty(graph.n, dtype=torch.float32, device="cuda") if want_sigma_s else None
    gg = torch.empty(graph.n, dtype=torch.float32, device="cuda") if want_g else None
    ga = torch.empty(n_vox, dtype=torch.float32, device="cuda") if voxel is not None else None
    check(_LIB.pg_propagate_adjoint(graph.handle, _ptr(dI), _ptr(first), first.numel(), spp, width, height,
                                    _ptr(gs), _ptr(gg), _ptr(voxel), _ptr(sigma_t), _ptr(ga), n_vox,
                                    int(recompute_weights), _stream_ptr(stream)), "pg_propagate_adjoint")
    return {"grad_sigma_s": gs, "grad_g": gg, "grad_albedo": ga}


def pg_prepare_adjoint(graph: Graph, stream=None) -> None:
    """Build the transposed weights for pg_propagate_adjoint on ``stream``
    (e.g. a side stream while pg_propagate runs); see include/pg.h."""
    check(_LIB.pg_prepare_adjoint(graph.handle, _stream_ptr(stream)), "pg_prepare_adjoint")


def pg_propagate_noalloc(graph: Graph, L0: torch.Tensor, iters: int, out: torch.Tensor, tol: float = 0.0,
                         stream=None) -> torch.Tensor:
    """pg_propagate without device allocation (scratch in a static device
    array; see include/pg.h). ``out`` must be preallocated by the caller."""
    check(_LIB.pg_propagate_noalloc(graph.handle, _ptr(L0), iters, tol, _ptr(out), _stream_ptr(stream)),
          "pg_propagate_noalloc")
    return out


def launch_count() -> int:
    """Kernels launched by libpg in this process (diagnostic)."""
    return int(_LIB.pg_launch_count())


from .solver import Solver  # noqa: E402

__all__ = ["Solver", "launch_count", "Vertices", "Graph", "PgError", "pg_build_graph", "pg_aggregate", "pg_propagate",
           "pg_gather", "pg_gather_ex", "extra_from_records", "pg_propagate_adjoint", "pg_propagate_noalloc",
           "pg_record", "pg_prepare_adjoint"]
