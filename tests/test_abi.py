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
