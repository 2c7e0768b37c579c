"""The C ABI library loads and exports every function include/pg.h declares.

No compute call is made (no GPU here): only argument checks that return
before any CUDA work.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]


def _declared():
    names = set()
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(pg_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    __graft_entry__._build_module().build()
    from paper_2404_11894_gb300 import _lib

    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"pg_build_graph", "pg_aggregate", "pg_propagate", "pg_gather", "pg_propagate_adjoint"} <= names
    for name in sorted(names):
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_binding_names_match_c(lib):
    import paper_2404_11894_gb300 as pg

    for name in ("pg_build_graph", "pg_aggregate", "pg_propagate", "pg_gather", "pg_propagate_adjoint"):
        assert callable(getattr(pg, name))


def test_argument_errors_without_gpu(lib):
    from paper_2404_11894_gb300._lib import PgBuildParams, PgVertices

    p = PgBuildParams()
    p.k = 0
    for a in range(3):
        p.bbox_lo[a] = 0.0
        p.bbox_hi[a] = 1.0
    out = ctypes.c_void_p()
    v = PgVertices()
    assert lib.pg_build_graph(ctypes.byref(v), 10, ctypes.byref(p), None, ctypes.byref(out)) == 6  # k=0
    p.k = 33
    assert lib.pg_build_graph(ctypes.byref(v), 10, ctypes.byref(p), None, ctypes.byref(out)) == 6
    p.k = 8
    assert lib.pg_build_graph(ctypes.byref(v), 10, ctypes.byref(p), None, ctypes.byref(out)) == 1  # NULL arrays
    assert lib.pg_build_graph(ctypes.byref(v), -1, ctypes.byref(p), None, ctypes.byref(out)) == 1
    p.bbox_hi[0] = 0.0
    assert lib.pg_build_graph(ctypes.byref(v), 0, ctypes.byref(p), None, ctypes.byref(out)) == 1  # empty box
    assert lib.pg_aggregate(None, None, 0, None, None, None) == 1
    assert lib.pg_propagate(None, None, None, 1, 0.0, 0, None, None, None, None) == 1
    assert lib.pg_gather(None, None, None, None, None, 0, 1, 0, 0, None, None) == 1
    assert lib.pg_gather_ex(None, None, None, None, None, 0, 1, 0, 0, None, None, None) == 1
    assert lib.pg_graph_release_weights(None) == 1
    lib.pg_graph_destroy(None)
    assert lib.pg_status_string(4) == b"non-finite input"


def test_host_step_and_shard_argument_errors_without_gpu(lib):
    """pg_step_host and the shard calls refuse bad arguments before any CUDA
    work; a host-only shard plan needs no device at all."""
    import numpy as np

    from paper_2404_11894_gb300._lib import PgShardInfo, PgStepParams, PgVertices

    prm = PgStepParams(k=8, iters=3, wdtype=0, spp=1, width=2, height=2, adjoint=0, n_vox=0)
    img = np.zeros(4, np.float32)
    ip = img.ctypes.data_as(ctypes.c_void_p)
    v = PgVertices()
    assert lib.pg_step_host(None, 0, None, None, None, 4, None, None, ctypes.byref(prm), ip, None, None, None) == 1
    assert lib.pg_step_host(ctypes.byref(v), 0, None, None, None, 5, None, None, ctypes.byref(prm), ip, None, None,
                            None) == 1  # paths != width * height * spp
    assert lib.pg_step_host(ctypes.byref(v), 10, None, None, None, 4, None, None, ctypes.byref(prm), ip, None, None,
                            None) == 1  # NULL records
    # a gradient needs a target
    first = np.full(4, -1, np.int32)
    fp = first.ctypes.data_as(ctypes.c_void_p)
    assert lib.pg_step_host(ctypes.byref(v), 0, None, fp, ip, 4, None, None, ctypes.byref(prm), ip, ip, None,
                            None) == 1
    out = ctypes.c_void_p()
    assert lib.pg_shard_create(None, 2, 0, None, ctypes.byref(out)) == 1
    col = np.array([[1, 3], [0, 2], [3, 3]], np.int32)  # 3 rows, zero slot 3
    cp = col.ctypes.data_as(ctypes.c_void_p)
    assert lib.pg_shard_create_host(cp, 3, 2, 3, 2, 2, ctypes.byref(out)) == 1   # shard out of range
    assert lib.pg_shard_create_host(cp, 3, 2, 2, 2, 0, ctypes.byref(out)) == 1   # zero slot inside the rows
    bad = np.array([[1, 7], [0, 2], [3, 3]], np.int32)
    assert lib.pg_shard_create_host(bad.ctypes.data_as(ctypes.c_void_p), 3, 2, 3, 2, 0, ctypes.byref(out)) == 1
    assert lib.pg_shard_create_host(cp, 3, 2, 3, 2, 1, ctypes.byref(out)) == 0
    info = PgShardInfo()
    assert lib.pg_shard_get_info(out, ctypes.byref(info)) == 0
    assert (info.n_shards, info.shard, info.row_end) == (2, 1, 3)
    # device calls on a host-only shard are refused
    assert lib.pg_shard_sweep(out, None, None, None) == 7
    lib.pg_shard_destroy(out)
