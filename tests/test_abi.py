"""The C-ABI library builds, loads and exports every symbol its header declares
(no GPU; no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            for m in re.finditer(r"^\s*(?:int|int64_t|void|const char\*)\s+(bfs_\w+)\s*\(", txt, flags=re.M):
                names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    import paper_1803_03922_gb300 as bfs

    lib = ctypes.CDLL(bfs.library_path())
    names = _declared()
    assert {"bfs_build_graph", "bfs_run", "bfs_free", "bfs_last_error"} <= names
    for name in names:
        assert hasattr(lib, name), name


def test_struct_layouts_match_binding():
    import paper_1803_03922_gb300 as bfs

    bfs._load()  # raises on any size mismatch


def test_options_default_and_errors_without_gpu():
    import paper_1803_03922_gb300 as bfs

    o = bfs.bfs_options_default()
    assert (o.th, o.alpha, o.beta, o.schedule, o.td_parent) == (64, 10, 18, 7, 1)
    assert o.barrier_timeout_ms == 2000
    h = ctypes.c_void_p()
    lib = bfs._load()
    # argument checks happen before any device call
    assert lib.bfs_build_graph(None, None, 0, 0, None, ctypes.byref(h), None) == bfs.BFS_ERR_INVALID
    assert "num_vertices" in bfs.bfs_last_error()
    assert lib.bfs_run(None, 0, None, None, None, None) == bfs.BFS_ERR_INVALID
    assert lib.bfs_run_many(None, None, 0, None, None, None, None) == bfs.BFS_ERR_INVALID
    lib.bfs_free(None)


def test_run_many_binding_checks_without_gpu():
    import numpy as np

    import paper_1803_03922_gb300 as bfs

    host = np.zeros(8, np.int32)
    with pytest.raises(ValueError):
        bfs.bfs_run_many(None, [1, 2], [host], [host, host])  # one buffer pair per source
    with pytest.raises(ValueError):
        bfs.bfs_run_many(None, [1], [host], [host], status=np.zeros(1, np.int64))
    with pytest.raises(bfs.BfsError):
        bfs.bfs_run_many(None, [], [], [])  # the library rejects a NULL graph


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1803_03922_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "oracle.h" not in txt and "liboracle" not in txt, f


def test_server_argument_checks_without_gpu():
    import paper_1803_03922_gb300 as bfs

    lib = bfs._load()
    o = bfs.bfs_server_options_default()
    assert (o.max_concurrent, o.max_lanes, o.with_parents) == (2, 64, 1)
    h = ctypes.c_void_p()
    for field, bad in (("max_lanes", 65), ("max_concurrent", 9), ("with_parents", 2), ("hbm_budget_bytes", -1)):
        o2 = bfs.bfs_server_options_default()
        setattr(o2, field, bad)
        assert lib.bfs_server_create(ctypes.byref(o2), ctypes.byref(h)) == bfs.BFS_ERR_INVALID, field
    t = ctypes.c_int64()
    assert lib.bfs_server_submit(None, 0, 0, None, None, 0, ctypes.byref(t)) == bfs.BFS_ERR_INVALID
    n = ctypes.c_int32()
    assert lib.bfs_server_poll(None, None, 0, 0, ctypes.byref(n)) == bfs.BFS_ERR_INVALID
    lib.bfs_server_destroy(None)
    assert bfs.bfs_server_now_ns() > 0
