"""Build of the CUDA libraries (sm_103a) next to their sources.

``libs3bfs.so`` is the product.  ``libs3bfs_checked.so`` is the same code
compiled with ``S3BFS_CHECKED=1``: every global index of the level step is
range-checked (an out-of-range one stops the traversal with BFS_E_CHECK
instead of an access), and ``bfs_run_frontiers`` dumps every level's
frontier.  nvcc compiles the kernels + C ABI (``csrc/s3bfs.cu``) and the
query server (``csrc/serve.cu``) of both, g++ the host CSR helpers
(``csrc/csr_host.cpp``), all in parallel; then nvcc links each shared library
with the CUDA runtime linked statically.  Objects go to ``_build/`` (ignored).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libs3bfs.so")
LIB_CHECKED = os.path.join(HERE, "libs3bfs_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = [os.path.join(CSRC, f) for f in ("s3bfs.cu", "level_loop.cuh", "s3bfs_device.cuh", "msbfs.cuh", "host_internal.h", "serve.cu", "serve_device.cuh", "csr_host.cpp")] + \
    [os.path.join(INCLUDE, "s3bfs.h")]
_lock = threading.Lock()


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is needed to build libs3bfs.so")


def _stale() -> bool:
    for lib in (LIB, LIB_CHECKED):
        if not os.path.exists(lib):
            return True
        t = os.path.getmtime(lib)
        if any(os.path.getmtime(s) > t for s in SOURCES):
            return True
    return False


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libs3bfs.so if missing or older than its sources; return its path."""
    with _lock:
        if not force and not _stale():
            return LIB
        os.makedirs(BUILD, exist_ok=True)
        nv = nvcc()
        nvflags = [nv, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
        ptx = ["-Xptxas", "-v"] if verbose else []
        obj = {k: os.path.join(BUILD, k + ".o") for k in ("s3bfs", "serve", "s3bfs_chk", "serve_chk", "csr_host")}
        chk = ["-DS3BFS_CHECKED=1"]
        cmds = [
            nvflags + ["-c", os.path.join(CSRC, "s3bfs.cu"), "-o", obj["s3bfs"]] + ptx,
            nvflags + ["-c", os.path.join(CSRC, "serve.cu"), "-o", obj["serve"]] + ptx,
            nvflags + chk + ["-c", os.path.join(CSRC, "s3bfs.cu"), "-o", obj["s3bfs_chk"]],
            nvflags + chk + ["-c", os.path.join(CSRC, "serve.cu"), "-o", obj["serve_chk"]],
            ["g++", "-O2", "-std=c++17", "-fPIC", "-I", INCLUDE, "-c", os.path.join(CSRC, "csr_host.cpp"), "-o",
             obj["csr_host"]],
        ]
        procs = [subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True) for c in cmds]
        outs = [p.communicate()[0] for p in procs]
        for c, p, o in zip(cmds, procs, outs):
            if p.returncode != 0:
                raise RuntimeError(f"build failed: {' '.join(c)}\n{o}")
            if verbose and o:
                print(o)
        for lib, objs in ((LIB, ("s3bfs", "serve", "csr_host")), (LIB_CHECKED, ("s3bfs_chk", "serve_chk", "csr_host"))):
            tmp = lib + f".tmp{os.getpid()}"
            link = [nv, *ARCH, "-shared", "-o", tmp] + [obj[k] for k in objs]
            r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"link failed: {' '.join(link)}\n{r.stdout}")
            os.replace(tmp, lib)
        return LIB
