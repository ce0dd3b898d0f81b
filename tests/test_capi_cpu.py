"""CPU-side checks of the C ABI: the library builds, loads, and exports
every function include/bfs.h declares; the binding declares the same set.
No compute calls (there is no GPU here)."""
from __future__ import annotations

import subprocess

import paper_2103_13577_gb300 as bfs
from paper_2103_13577_gb300 import _lib


def test_library_exports_every_declared_function():
    lib = bfs.load()
    declared = _lib.header_functions()
    assert "bfs_run" in declared and "bfs_submit" in declared and "bfs_poll" in declared
    for name in declared:
        assert hasattr(lib, name), f"{name} missing from libbfs.so"
    out = subprocess.check_output(["nm", "-D", "--defined-only", _lib.LIB_PATH], text=True)
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert set(declared) <= exported


def test_binding_covers_header():
    assert set(_lib.header_functions()) == set(_lib.SIGNATURES)


def test_status_strings_and_version():
    lib = bfs.load()
    assert lib.bfs_version() >= 100
    assert lib.bfs_status_string(bfs.BFS_ERR_TIMEOUT) == b"device wait timed out"
    assert lib.bfs_status_string(0) == b"ok"


def test_null_arguments_are_rejected_without_a_gpu():
    lib = bfs.load()
    assert lib.bfs_run(None, 0, None, None, None, 0) == bfs.BFS_ERR_INVALID_ARG
    assert lib.bfs_graph_free(None) == bfs.BFS_ERR_INVALID_ARG
    assert lib.bfs_poll(None, 1) == bfs.BFS_ERR_INVALID_ARG
    assert b"null" in lib.bfs_last_error()


def test_paths_arguments_are_checked_without_a_gpu():
    lib = bfs.load()
    # no context, offsets or outputs: refused before any CUDA call
    assert lib.bfs_run_paths(None, None, None, None, 4, 3, 0, 0, 0, None, None, None,
                             None) == bfs.BFS_ERR_INVALID_ARG
    assert b"paths" in lib.bfs_last_error()
