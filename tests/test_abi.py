"""The C ABI without a GPU: the library builds for sm_103a, loads, exports every
function include/grape_walk.h declares, its ctypes mirrors match the C struct
layouts, and argument errors come back before any CUDA call."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2110_06196_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "grape_walk.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(grape_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    return _lib.load()


def test_library_builds_for_sm103a(lib):
    assert os.path.exists(build.LIB)
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_every_declared_function_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 25
    for name in names:
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (grape_\w+)", out))
    assert set(names) <= exported


def test_binding_covers_every_declaration():
    assert set(declared_functions()) == set(_lib.SIGNATURES)


STRUCTS = {
    "grape_graph_info_t": _lib.GraphInfo,
    "grape_tuning_t": _lib.Tuning,
    "grape_walk_request_t": _lib.WalkRequest,
    "grape_walk_counters_t": _lib.Counters,
    "grape_server_config_t": _lib.ServerConfig,
    "grape_server_stats_t": _lib.ServerStats,
    "grape_ef_info_t": _lib.EFInfo,
    "grape_ef_counters_t": _lib.EFCounters,
}


def test_struct_layouts_match_header(tmp_path):
    lines = ["#include <stdio.h>", "#include <stddef.h>", f'#include "{HEADER}"', "int main(void){"]
    for cname, py in STRUCTS.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines.append("return 0;}")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", str(c), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n"):
        if line:
            s, f, v = line.split()
            got[(s, f)] = int(v)
    for cname, py in STRUCTS.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for field, _ in py._fields_:
            assert got[(cname, field)] == getattr(py, field).offset, (cname, field)


def test_status_strings(lib):
    for code in _lib.STATUS:
        s = lib.grape_status_string(code)
        assert isinstance(s, bytes) and len(s) > 0


def test_argument_errors_return_before_cuda(lib):
    INVALID = _lib.CODES["GRAPE_ERR_INVALID_ARG"]
    h = ctypes.c_void_p()
    # missing offsets, bad sizes, unknown flags
    assert lib.grape_graph_create(None, None, None, 10, 0, 0, None, ctypes.byref(h)) == INVALID
    assert lib.grape_graph_create(ctypes.c_void_p(8), None, None, 0, 0, 0, None,
                                  ctypes.byref(h)) == INVALID
    assert lib.grape_graph_create(ctypes.c_void_p(8), ctypes.c_void_p(8), None, 4, 4, 1 << 7,
                                  None, ctypes.byref(h)) == INVALID
    assert lib.grape_graph_create(ctypes.c_void_p(8), None, None, 4, 4, 0, None,
                                  ctypes.byref(h)) == INVALID
    # null graph / null out
    assert lib.grape_walks(None, None, 1, 4, 1, 1.0, 1.0, 0, None, None) == INVALID
    assert lib.grape_walks_batched(None, None, 0, None) == INVALID
    assert lib.grape_graph_info(None, None) == INVALID
    assert lib.grape_walk_server_create(None, None, ctypes.byref(h)) == INVALID
    assert lib.grape_walk_server_inject_fault(None, 0) == INVALID
    assert lib.grape_trim_scratch(-1) == INVALID
    assert lib.grape_philox4x32_10(None, -1, None, None) == INVALID
    assert lib.grape_sector_probe(None, 0, 0, 0, 0, 32, 8, 0, None, None, None, None) == INVALID
    # shapes outside the compiled (width, loads in flight) pairs, negative blocks
    for width, loads, blocks in ((32, 32, 0), (8, 8, 0), (4, 4, 0), (16, 64, 0), (32, 8, -1)):
        assert lib.grape_sector_probe(ctypes.c_void_p(256), 1 << 20, 1 << 10, 0, 0, width, loads,
                                      blocks, ctypes.c_void_p(256), None, None, None) == INVALID
    assert lib.grape_contexts_from_rows(None, 4, 8, 2, None, None) == INVALID
    for window in (0, 65):
        assert lib.grape_contexts_from_rows(ctypes.c_void_p(16), 4, 8, window,
                                            ctypes.c_void_p(16), None) == INVALID
    assert lib.grape_walk_contexts(None, None, 4, 8, 1, 1.0, 1.0, 0, 2, 0, 4, None, None,
                                   None) == INVALID
    assert lib.grape_walks_approx(None, None, 4, 8, 1, 1.0, 1.0, 0, -1, None, None) == INVALID
    assert lib.grape_walks_approx(None, None, 4, 8, 1, 1.0, 1.0, 0, 3, None, None) == INVALID
    # Elias-Fano store: bad sizes, quanta that are not powers of two, null store
    for quantum in (0, 3, 1 << 17):
        assert lib.grape_ef_graph_create(ctypes.c_void_p(8), ctypes.c_void_p(8), None, 4, 4,
                                         quantum, 0, None, ctypes.byref(h)) == INVALID
    assert lib.grape_ef_graph_create(None, None, None, 4, 0, 64, 0, None, ctypes.byref(h)) == INVALID
    assert lib.grape_ef_graph_create(ctypes.c_void_p(8), None, None, 4, 4, 64, 0, None,
                                     ctypes.byref(h)) == INVALID
    assert lib.grape_ef_graph_create(ctypes.c_void_p(8), ctypes.c_void_p(8), None, 4, 1 << 40,
                                     64, 0, None, ctypes.byref(h)) == INVALID
    assert lib.grape_ef_walks(None, None, 4, 8, 1, 1.0, 1.0, 0, 4096, None, None) == INVALID
    assert lib.grape_ef_select(None, None, 1, None, None) == INVALID
    assert lib.grape_ef_rank(None, None, 1, None, None) == INVALID
    assert lib.grape_ef_graph_info(None, None) == INVALID
    assert lib.grape_walks_cumsum(None, None, 4, 8, 1, 1.0, 1.0, 0, None, None) == INVALID
    lib.grape_ef_graph_destroy(None)
    lib.grape_graph_destroy(None)
    lib.grape_walk_server_destroy(None)
    lib.grape_batch_plan_destroy(None)
