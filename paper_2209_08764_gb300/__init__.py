"""S3BFS level step on GB300 (sm_103a) behind a C ABI.

``binding`` exposes the C functions one to one (``bfs_create_csr``,
``bfs_run``, ``bfs_run_batch``, ``bfs_destroy``, ...).  :class:`BFSGraph` is a
small convenience wrapper that keeps outputs in torch CUDA tensors; PyTorch is
used only for device memory and the current stream.
"""
from __future__ import annotations

from .binding import (BFS_DEBUG_STALL_BARRIER, BFS_DEDUP, BFS_DEVICE_PTRS, BFS_E_CUDA, BFS_E_INVAL,  # noqa: F401
                      BFS_E_MULTIGRAPH, BFS_E_NOMEM, BFS_E_TIMEOUT, BFS_LEVEL_FIELDS, BFS_OK, BFS_SYMMETRIC, BFS_VALIDATE,
                      BFSError, bfs_create_csr, bfs_destroy, bfs_graph_info, bfs_last_error, bfs_opts, bfs_run,
                      bfs_run_batch, bfs_stats, bfs_strerror)


def build(force: bool = False, verbose: bool = False) -> str:
    from . import _build
    return _build.build(force=force, verbose=verbose)


class BFSGraph:
    """One CSR graph resident on the current CUDA device.

    ``row_ptr`` / ``col_idx``: int32 CSR as numpy arrays or torch tensors (host
    or CUDA).  Outputs of :meth:`run` are int32 CUDA tensors unless host
    arrays are passed in.
    """

    def __init__(self, row_ptr, col_idx, flags: int = BFS_VALIDATE, opts: bfs_opts | None = None,
                 stream=None):
        import torch
        self.n = int(len(row_ptr) - 1)
        self.nnz = int(len(col_idx))
        if isinstance(row_ptr, torch.Tensor) and row_ptr.is_cuda:
            flags |= BFS_DEVICE_PTRS
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.handle = bfs_create_csr(self.n, self.nnz, row_ptr, col_idx, flags, opts,
                                     self.stream.cuda_stream)
        self.info = bfs_graph_info(self.handle)

    def run(self, src: int, level=None, parent=None, want_parent: bool = True, per_level_cap: int = 0):
        """One traversal; returns (level, parent or None, stats dict)."""
        import ctypes

        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        if level is None:
            level = torch.empty(self.n, dtype=torch.int32, device=dev)
        if parent is None and want_parent:
            parent = torch.empty(self.n, dtype=torch.int32, device=dev)
        st = bfs_stats()
        buf = None
        if per_level_cap > 0:
            buf = (ctypes.c_int32 * (per_level_cap * BFS_LEVEL_FIELDS))()
            st.per_level = ctypes.cast(buf, ctypes.POINTER(ctypes.c_int32))
            st.per_level_cap = per_level_cap
        bfs_run(self.handle, src, level, parent, st)
        out = {f: getattr(st, f) for f, _ in bfs_stats._fields_ if f not in ("per_level", "per_level_cap")}
        if buf is not None:
            L = min(st.num_levels, per_level_cap)
            out["per_level"] = [list(buf[i * BFS_LEVEL_FIELDS:(i + 1) * BFS_LEVEL_FIELDS]) for i in range(L)]
        return level, parent, out

    def close(self):
        if getattr(self, "handle", None):
            bfs_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
