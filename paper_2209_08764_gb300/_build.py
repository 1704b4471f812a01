"""Build of the CUDA library ``libs3bfs.so`` (sm_103a) next to its sources.

nvcc compiles the kernels + C ABI (``csrc/s3bfs.cu``) and the query server
(``csrc/serve.cu``), g++ the host CSR helpers (``csrc/csr_host.cpp``), all in
parallel; then nvcc links a shared library with the CUDA runtime linked
statically.  Objects go to ``_build/`` (ignored).
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
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in SOURCES)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libs3bfs.so if missing or older than its sources; return its path."""
    with _lock:
        if not force and not _stale():
            return LIB
        os.makedirs(BUILD, exist_ok=True)
        nv = nvcc()
        obj_cu = os.path.join(BUILD, "s3bfs.o")
        obj_serve = os.path.join(BUILD, "serve.o")
        obj_cpp = os.path.join(BUILD, "csr_host.o")
        nvflags = [nv, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
        cmds = [
            nvflags + ["-c", os.path.join(CSRC, "s3bfs.cu"), "-o", obj_cu] + (["-Xptxas", "-v"] if verbose else []),
            nvflags + ["-c", os.path.join(CSRC, "serve.cu"), "-o", obj_serve] + (["-Xptxas", "-v"] if verbose else []),
            ["g++", "-O2", "-std=c++17", "-fPIC", "-I", INCLUDE, "-c", os.path.join(CSRC, "csr_host.cpp"), "-o",
             obj_cpp],
        ]
        procs = [subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True) for c in cmds]
        outs = [p.communicate()[0] for p in procs]
        for c, p, o in zip(cmds, procs, outs):
            if p.returncode != 0:
                raise RuntimeError(f"build failed: {' '.join(c)}\n{o}")
            if verbose and o:
                print(o)
        tmp = LIB + f".tmp{os.getpid()}"
        link = [nv, *ARCH, "-shared", "-o", tmp, obj_cu, obj_serve, obj_cpp]
        r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed: {' '.join(link)}\n{r.stdout}")
        os.replace(tmp, LIB)
        return LIB
