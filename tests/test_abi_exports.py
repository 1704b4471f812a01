"""The C-ABI library builds, loads, and exports every function that
include/s3bfs.h declares (CPU only: no kernel is launched)."""
import ctypes
import os
import re

import pytest

import paper_2209_08764_gb300 as pkg
from paper_2209_08764_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(bfs_\w+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    pkg.build()
    return B.load()


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert {"bfs_create_csr", "bfs_run", "bfs_run_batch", "bfs_destroy", "bfs_strerror"} <= declared
    for name in sorted(declared):
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    assert set(B.EXPORTS) >= declared


def test_checked_build_exports_the_same_symbols():
    from paper_2209_08764_gb300 import _build
    pkg.build()
    chk = ctypes.CDLL(_build.LIB_CHECKED)
    for name in sorted(_declared()):
        assert hasattr(chk, name), f"{name} missing from the checked build"
    chk.bfs_strerror.restype = ctypes.c_char_p
    assert b"checked build" in chk.bfs_strerror(B.BFS_E_CHECK)


def test_frontier_dump_needs_the_checked_build(lib):
    # the production library refuses before touching the (NULL) graph
    assert lib.bfs_run_frontiers(None, 0, None, None, None, None) == B.BFS_E_INVAL
    assert "checked build" in B.bfs_last_error()


def test_host_only_calls(lib):
    assert B.bfs_strerror(0) == "ok"
    assert "timed out" in B.bfs_strerror(B.BFS_E_TIMEOUT)
    assert B.bfs_strerror(12345) == "unknown error"
    # argument checks happen before any CUDA call
    out = ctypes.c_void_p()
    assert lib.bfs_create_csr(0, 0, None, None, 0, None, None, ctypes.byref(out)) == B.BFS_E_INVAL
    assert out.value is None
    assert "n = 0" in B.bfs_last_error()
    assert lib.bfs_run(None, 0, None, None, None) == B.BFS_E_INVAL
    assert lib.bfs_run_batch(None, None, 0, None, None, None) == B.BFS_E_INVAL
    lib.bfs_destroy(None)


_STRUCTS = ("bfs_opts", "bfs_stats", "bfs_server_opts", "bfs_completion")


def _c_layout(tmp_path):
    """sizeof and offsetof of every field, as the C compiler lays the header's
    structs out (gcc, host ABI)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "s3bfs.h"', "int main(void) {"]
    for st in _STRUCTS:
        lines.append(f'  printf("{st} size %zu\\n", sizeof({st}));')
        for name, _ in getattr(B, st)._fields_:
            lines.append(f'  printf("{st} {name} %zu\\n", offsetof({st}, {name}));')
    lines.append("  return 0;\n}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)], text=True)
    return {tuple(l.split()[:2]): int(l.split()[2]) for l in out.splitlines()}


def test_struct_layout_matches_header(tmp_path):
    c = _c_layout(tmp_path)
    for st in _STRUCTS:
        py = getattr(B, st)
        assert c[(st, "size")] == ctypes.sizeof(py), st
        for name, _ in py._fields_:
            assert c[(st, name)] == getattr(py, name).offset, (st, name)
    # the header's field lists and the binding's agree in full
    hdr = open(os.path.join(ROOT, "include", "s3bfs.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    for st in _STRUCTS:
        body = re.search(r"typedef struct " + st + r"\s*\{(.*?)\}\s*" + st + ";", hdr, re.S).group(1)
        names = []
        for decl in body.split(";"):
            decl = decl.strip()
            if decl:
                first, *rest = decl.split(",")
                names += [first.split()[-1].lstrip("*")] + [r.strip().lstrip("*") for r in rest]
        assert names == [n for n, _ in getattr(B, st)._fields_], st
