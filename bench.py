"""Benchmark of the S3BFS level step: GTEPS and HBM roofline fraction.

Default workload: R-MAT scale 22, edgefactor 16 (A/B/C/D = 0.57/0.19/0.19/0.05,
symmetrised, self-loops and duplicates removed, int32 CSR), 64 seeded
non-isolated sources traversed one at a time.  One step = the 64 traversals;
``value`` = traversed edges (Graph500 count: half the degree sum of the reached
vertices) of all steps and ranks / the slowest rank's device time.

Prints one JSON line.  ``--impl reference`` times the CPU oracle (sequential
FIFO BFS, one core) on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import csv
import ctypes
import hashlib
import io
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import graphgen  # noqa: E402

METRIC = "BFS GTEPS + HBM roofline fraction at RMAT s22; served-query p50/p99 latency"
L2_BYTES = 129 * 1024 * 1024
FALLBACK_HBM_GBS = 6800.0

WORKLOADS = {
    "rmat22": dict(kind="rmat", scale=22, edgefactor=16, seed=1, sources=64, src_seed=2),
    "rmat16": dict(kind="rmat", scale=16, edgefactor=16, seed=1, sources=64, src_seed=2),
    "er20": dict(kind="er", n=1 << 20, m=8 << 20, seed=4, sources=64, src_seed=2),
    "grid4096": dict(kind="grid", rows=4096, cols=4096, p=0.01, seed=3, sources=8, src_seed=3),
}


def make_graph(w):
    if w["kind"] == "rmat":
        return graphgen.rmat(w["scale"], w["edgefactor"], seed=w["seed"])
    if w["kind"] == "er":
        return graphgen.erdos_renyi(w["n"], w["m"], seed=w["seed"])
    return graphgen.grid(w["rows"], w["cols"], w["p"], seed=w["seed"])


def sources_for(w, rp, rank):
    from paper_2209_08764_gb300.replicas import rank_source_seed
    src = graphgen.sample_sources(rp, w["sources"], seed=rank_source_seed(w["src_seed"], rank))
    if w["kind"] == "grid" and rank == 0:
        src = np.concatenate([[0], src[:-1]]).astype(np.int32)   # the corner: maximum depth
    return src


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def strip_c_comments(src: str) -> str:
    """C/C++ source without comments and with whitespace runs collapsed, so
    that an edit of comments alone leaves the hash below unchanged."""
    import re
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    return " ".join(src.split())


KERNEL_SOURCES = {
    "level_loop": ("paper_2209_08764_gb300/csrc/level_loop.cuh", "paper_2209_08764_gb300/csrc/s3bfs_device.cuh"),
    "msbfs": ("paper_2209_08764_gb300/csrc/msbfs.cuh", "paper_2209_08764_gb300/csrc/s3bfs_device.cuh"),
}


def kernel_source_hash(kernel="level_loop"):
    """First 16 hex digits of the sha256 of a kernel's device sources (the
    kernel and its building blocks, comments stripped): the key under which
    a committed ncu summary is valid.  Host code is not part of it."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, f), encoding="utf-8") as fh:
            h.update(strip_c_comments(fh.read()).encode())
    return h.hexdigest()[:16]


def profiled(workload, key="dram_bytes_per_launch", name="level_loop", kernel="level_loop"):
    """A per-launch counter from the committed ncu summary
    profiles/<name>_<workload>.json, if it was taken on the current kernel
    source; else None."""
    path = os.path.join(ROOT, "profiles", f"{name}_{workload}.json")
    try:
        with open(path) as f:
            p = json.load(f)
    except (OSError, ValueError):
        return None
    if p.get("kernel_source_sha256_16") != kernel_source_hash(kernel):
        return None
    return p.get(key)


def profiled_traffic(workload, name="level_loop", kernel="level_loop"):
    """DRAM bytes per launch of a kernel (ncu), or None."""
    return profiled(workload, "dram_bytes_per_launch", name, kernel)


def gather_peak(torch, dev):
    """Measured rate of isolated 4-byte loads at random addresses: torch's
    gather kernel reading an int32 table of 16 MiB (L2-resident, like the
    level array the explore tests) and of 1 GiB (HBM), with 2^27 random
    indices each; the higher rate, in loads (sectors) per second.  A
    reference rate for a kernel whose every test is one scattered load, not
    a hard ceiling: the gather also streams 12 B of index and output per
    load, and the level step's biggest level runs above it."""
    best = 0.0
    g = torch.Generator(device=dev).manual_seed(7)
    out = torch.empty(1 << 27, dtype=torch.int32, device=dev)
    for size in (1 << 22, 1 << 28):
        table = torch.zeros(size, dtype=torch.int32, device=dev)
        idx = torch.randint(0, size, (1 << 27,), generator=g, device=dev, dtype=torch.int64)
        for _ in range(3):
            torch.index_select(table, 0, idx, out=out)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(10):
            torch.index_select(table, 0, idx, out=out)
        e1.record()
        torch.cuda.synchronize()
        best = max(best, 10 * idx.numel() / (e0.elapsed_time(e1) / 1e3))
        del table, idx
    del out
    return best


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out = self.proc.communicate(timeout=5)[0]
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out = self.proc.communicate()[0]

    def summary(self):
        rows = [r for r in csv.reader(io.StringIO(getattr(self, "out", ""))) if len(r) >= 9]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip().lower() == "active"})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows)}


class EnergyMeter:
    """GPU energy from NVML's total-energy counter (millijoules since the
    driver loaded), read through ctypes; every reading is None where NVML is
    not available.  Reading the counter changes nothing on the GPU."""

    def __init__(self, torch, dev):
        self.lib = None
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return
            h = ctypes.c_void_p()
            bus = getattr(torch.cuda.get_device_properties(dev), "pci_bus_id", None)
            dom = getattr(torch.cuda.get_device_properties(dev), "pci_domain_id", 0)
            ok = False
            if bus is not None:
                key = f"{dom:08x}:{bus:02x}:00.0".encode()
                ok = lib.nvmlDeviceGetHandleByPciBusId_v2(key, ctypes.byref(h)) == 0
            if not ok and lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(dev), ctypes.byref(h)) != 0:
                return
            self.lib, self.h = lib, h
        except (OSError, AttributeError):
            self.lib = None

    def read_mj(self):
        if self.lib is None:
            return None
        e = ctypes.c_ulonglong()
        return e.value if self.lib.nvmlDeviceGetTotalEnergyConsumption(self.h, ctypes.byref(e)) == 0 else None


def energy_per_traversal(meter, run_one, srcs, seconds=0.6, repeats=3):
    """Joules per traversal and mean power: NVML's energy counter around
    >= seconds of back-to-back traversals of the sources, repeated; the mean
    and the standard deviation over the repeats."""
    import torch
    if meter is None or meter.read_mj() is None:
        return None
    j, w, ks = [], [], []
    for _ in range(repeats):
        torch.cuda.synchronize()
        e0, t0, k = meter.read_mj(), time.perf_counter(), 0
        while time.perf_counter() - t0 < seconds:
            for s in srcs:
                run_one(int(s))
                k += 1
        torch.cuda.synchronize()
        e1, t1 = meter.read_mj(), time.perf_counter()
        if e1 is None or e1 <= e0:
            return None
        j.append((e1 - e0) * 1e-3 / k)
        w.append((e1 - e0) * 1e-3 / (t1 - t0))
        ks.append(k)
    return {"j_per_traversal": float(np.mean(j)), "j_per_traversal_std": float(np.std(j, ddof=1)),
            "avg_w": float(np.mean(w)), "repeats": repeats, "traversals": int(sum(ks)),
            "seconds_per_repeat": seconds, "source": "NVML total energy counter"}


def sms_total(torch, dev):
    return torch.cuda.get_device_properties(dev).multi_processor_count


def active_sms_summary(rows, sms):
    """Active SMs per level of one traversal (the first source's per-level
    records: SMs hosting at least one warp with a chunk); the rest of the SMs
    are parked at the grid barrier for that level."""
    a = np.asarray(rows)[:, 4].astype(np.int64) if rows is not None and len(rows) else np.zeros(0, np.int64)
    if len(a) == 0:
        return None
    out = {"sms": int(sms), "mean": round(float(a.mean()), 2), "levels_on_one_sm": int((a <= 1).sum()),
           "levels": int(len(a))}
    if len(a) <= 64:
        out["per_level"] = a.tolist()
    return out


def ratio_with_error(a, b):
    """a / b of two energy records, with the standard deviation propagated from
    the repeats of each (first order)."""
    if not a or not b or not a.get("j_per_traversal") or not b.get("j_per_traversal"):
        return None
    r = a["j_per_traversal"] / b["j_per_traversal"]
    ra = a.get("j_per_traversal_std", 0.0) / a["j_per_traversal"]
    rb = b.get("j_per_traversal_std", 0.0) / b["j_per_traversal"]
    return {"ratio": round(r, 4), "std": round(r * (ra * ra + rb * rb) ** 0.5, 4)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args, w):
    """The CPU oracle as the reference arm: sequential BFS, one core."""
    import oracle
    ws, rank, _ = dist_setup()
    if rank != 0:
        return
    rp, ci = make_graph(w)
    srcs = sources_for(w, rp, 0)
    orc = oracle.Oracle(rp, ci)
    per_step = args.ref_sources
    level = np.empty(len(rp) - 1, np.int32)
    parent = np.empty(len(rp) - 1, np.int32)
    edges = 0
    t_total = 0.0
    k = 0
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        e = 0
        for j in range(per_step):
            s = int(srcs[k % len(srcs)])
            k += 1
            orc.bfs(s, level, parent)
            e += oracle.traversed_edges(rp, level)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            t_total += dt
            edges += e
    gteps = edges / t_total / 1e9
    sample = f"{per_step} of the {len(srcs)} sources per step, one traversal each"
    line = {"metric": METRIC, "value": gteps, "unit": "GTEPS", "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": config_of(args.workload, w, rp, ci),
            "cpu_baseline": {"value": gteps, "unit": "GTEPS", "cores": 1, "kind": "oracle", "sample": sample,
                             "host": host_info()},
            "e2e": {"value": gteps, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def graph500_edges(deg, level, st) -> int:
    """Traversed edges of one traversal, Graph500 count for a symmetric CSR:
    half the summed degree of the reached vertices.  The library sums the
    same degrees on the device (``edges_scanned`` = sum of e_l over the
    levels); the two counts must agree, so the GPU arm's numerator is the
    definition the tests pin on the CPU side."""
    host = int(deg[np.asarray(level) >= 0].sum() // 2)
    dev = int(st.edges_scanned) // 2
    if host != dev:
        raise RuntimeError(f"traversed-edge counts disagree: degree sum {host}, library {dev}")
    return dev


def config_of(name, w, rp, ci):
    c = {"workload": name, "n": int(len(rp) - 1), "nnz": int(len(ci)), "sources": int(w["sources"])}
    c.update({k: v for k, v in w.items() if k not in ("kind", "sources")})
    c["l2"] = f"inputs larger than L2: CSR {(4 * (len(rp) + len(ci))) / 2**20:.0f} MiB vs L2 129 MiB" \
        if 4 * (len(rp) + len(ci)) > L2_BYTES else "CSR smaller than L2 (no flush)"
    c["parallelism"] = "replicas"
    return c


def cpu_baseline(w, rp, ci, srcs, budget_s):
    import oracle
    orc = oracle.Oracle(rp, ci)
    level = np.empty(len(rp) - 1, np.int32)
    parent = np.empty(len(rp) - 1, np.int32)
    edges, t, k = 0, 0.0, 0
    while k < len(srcs) and (t < budget_s or k < 1):
        t0 = time.perf_counter()
        orc.bfs(int(srcs[k]), level, parent)
        t += time.perf_counter() - t0
        edges += oracle.traversed_edges(rp, level)
        k += 1
    return {"value": edges / t / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
            "sample": f"first {k} of the {len(srcs)} sources, one traversal each ({t:.1f} s)",
            "host": host_info()}


def host_info():
    """CPU model and logical cores of the host the CPU baseline ran on."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware") and ":" in line:
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    import platform
    return {"cpu": model or platform.processor() or platform.machine(), "nproc": os.cpu_count(),
            "machine": platform.machine()}


def parse_cpulist(spec):
    """'0-3,8,10-11' -> [0, 1, 2, 3, 8, 10, 11]"""
    cpus = []
    for part in spec.strip().split(","):
        if not part:
            continue
        a, _, b = part.partition("-")
        cpus.extend(range(int(a), int(b or a) + 1))
    return cpus


def bind_gpu_local_cpus(torch, dev):
    """Pin this process to the CPUs of the GPU's own NUMA node (sysfs
    local_cpulist of its PCI function), so that pinned host buffers come from
    the memory closest to the GPU.  Returns the CPU list, or None where the
    system does not say (nothing changes then)."""
    try:
        prop = torch.cuda.get_device_properties(dev)
        addr = "%04x:%02x:%02x.0" % (getattr(prop, "pci_domain_id", 0), prop.pci_bus_id,
                                     getattr(prop, "pci_device_id", 0))
        with open(f"/sys/bus/pci/devices/{addr}/local_cpulist") as f:
            spec = f.read().strip()
        cpus = [c for c in parse_cpulist(spec) if c in os.sched_getaffinity(0)]
        if not cpus:
            return None
        os.sched_setaffinity(0, cpus)
        return spec
    except (OSError, ValueError, AttributeError):
        return None


def run_batch_mode(args, w, rp, ci, srcs, B, torch, dist, ws, rank, dev, replicas):
    """One step = one bfs_run_batch over all sources (groups of 64 share a
    bitmask traversal); compared with the same sources run one at a time."""
    line = measure_batch(args, w, rp, ci, srcs, B, torch, dist, ws, rank, dev, replicas)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def measure_batch(args, w, rp, ci, srcs, B, torch, dist, ws, rank, dev, replicas):
    """The bitmask batch's line (rank 0; None elsewhere)."""
    n, nnz = len(rp) - 1, len(ci)
    k = len(srcs)
    stream = torch.cuda.current_stream()
    g = B.bfs_create_csr(n, nnz, rp, ci, B.BFS_VALIDATE | B.BFS_SYMMETRIC, None, stream.cuda_stream)
    L = torch.empty(k * n, dtype=torch.int32, device=dev)
    P = None if args.no_parents else torch.empty(k * n, dtype=torch.int32, device=dev)
    S = np.ascontiguousarray(srcs, np.int32)
    st = (B.bfs_stats * k)()
    for _ in range(args.warmup):
        B.bfs_run_batch(g, S, k, L, P, None)
    B.bfs_run_batch(g, S, k, L, P, st)
    deg = np.diff(rp.astype(np.int64))
    Lh = L.cpu().numpy().reshape(k, n)
    teps = [graph500_edges(deg, Lh[i], st[i]) for i in range(k)]
    edges_per_step = sum(teps)
    levels = max(st[i].num_levels for i in range(k))
    work = st[0].work_edges
    # enough steps for the clock sampler (100 ms period) to see the timed region
    torch.cuda.synchronize()
    t_one = time.perf_counter()
    B.bfs_run_batch(g, S, k, L, P, None)
    torch.cuda.synchronize()
    t_one = time.perf_counter() - t_one
    steps = max(args.steps, int(np.ceil(0.4 / max(t_one, 1e-6))))
    if dist:
        # every rank times the same number of steps
        t = torch.tensor([steps], device=torch.device("cuda", dev))
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        steps = int(t.item())
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms_kernel = []
    with ClockSampler(dev) as clk:
        ev0.record(stream)
        for _ in range(steps):
            B.bfs_run_batch(g, S, k, L, P, st)
            ms_kernel.append(st[0].ms_level_step)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    ms_max, total_edges = replicas.aggregate(dist, ms, edges_per_step * steps,
                                             torch.device("cuda", dev) if dist else None)
    gteps = total_edges / (ms_max / 1e3) / 1e9
    # the same sources one at a time through bfs_run (single-source S3BFS)
    lv = torch.empty(n, dtype=torch.int32, device=dev)
    pa = torch.empty(n, dtype=torch.int32, device=dev)
    for s in S[:2]:
        B.bfs_run(g, int(s), lv, pa, None)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s in S:
        B.bfs_run(g, int(s), lv, pa, None)
    e1.record(stream)
    torch.cuda.synchronize()
    seq_gteps = edges_per_step / (e0.elapsed_time(e1) / 1e3) / 1e9
    peak, peak_kind = peaks()
    kms = float(np.mean(ms_kernel))
    # pull: 12 B per pulled edge (col_idx + the neighbour's frontier mask) and
    # 24 B per vertex per level (seen read + write, next frontier mask); the
    # k x n levels (and parents) written once
    k_out = 8 if P is not None else 4
    bytes_launch = 12.0 * work + 24.0 * n * levels + k_out * k * n
    achieved = bytes_launch / (kms / 1e3) / 1e9
    if rank == 0:
        line = {"metric": METRIC, "value": round(gteps, 3), "unit": "GTEPS", "n_gpus": ws, "steps": steps,
                "warmup": args.warmup, "ms_per_step": ms_max / steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
                "config": dict(config_of(args.workload, w, rp, ci), mode="batch-bitmask", k=k,
                               parents=not args.no_parents),
                "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                             "frac": round(achieved / peak, 4),
                             "traffic": profiled_traffic(args.workload, "msbfs", "msbfs") if P is not None else None,
                             "peak_kind": peak_kind,
                             "kernel": "k_msbfs", "algorithmic_bytes_per_launch": bytes_launch,
                             "avg_launch_ms": kms, "model": "12 B per pulled edge + 24 B per vertex per level + 4 B (8 with parents) "
                                      "per (source, vertex) output"},
                "clocks": clk.summary(), "gpu_launches": int(steps * st[0].launches * ((k + 63) // 64)),
                "sequential_gteps": round(seq_gteps, 3), "batch_speedup": round(gteps / seq_gteps, 2),
                "levels": levels, "pulled_edges": int(work)}
    else:
        line = None
    B.bfs_destroy(g)
    return line


def torch_device_index():
    import torch
    return torch.cuda.current_device()


def serving_pool():
    """The 32-graph serving pool: R-MAT s12..s22 (11), ER mean degree 8 with
    n = 2^12..2^22 (11), 4-neighbour grids 256^2..2048^2 with 1% of edges
    deleted (7), R-MAT s14/s16/s18 with a second seed (3)."""
    pool = []
    for sc in range(12, 23):
        pool.append((f"rmat{sc}", lambda sc=sc: graphgen.rmat(sc, 16, seed=1)))
    for lg in range(12, 23):
        pool.append((f"er{lg}", lambda lg=lg: graphgen.erdos_renyi(1 << lg, 4 << lg, seed=4)))
    for side in (256, 362, 512, 724, 1024, 1448, 2048):
        pool.append((f"grid{side}", lambda side=side: graphgen.grid(side, side, 0.01, seed=3)))
    for sc in (14, 16, 18):
        pool.append((f"rmat{sc}b", lambda sc=sc: graphgen.rmat(sc, 16, seed=2)))
    return pool


def run_serve_mode(args, B, torch):
    """Continuous-batching server over the pool vs the same stream served one
    query at a time by bfs_run (first come, first served)."""
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    t_gen = time.perf_counter()
    pool = serving_pool()
    graphs, handles, degs, nonisolated = [], [], [], []
    for name, make in pool:
        rp, ci = make()
        h = B.bfs_create_csr(len(rp) - 1, len(ci), rp, ci, 0, None, stream.cuda_stream)
        graphs.append((name, len(rp) - 1, len(ci)))
        handles.append(h)
        d = np.diff(rp.astype(np.int64))
        degs.append(d)
        nonisolated.append(np.nonzero(d > 0)[0].astype(np.int32))
    t_gen = time.perf_counter() - t_gen
    rng = np.random.default_rng(5)
    N = args.serve_queries
    gsel = rng.integers(0, len(pool), size=N)
    srcs = np.array([nonisolated[g][rng.integers(len(nonisolated[g]))] for g in gsel], np.int32)
    # service time of every query alone (plain single-source S3BFS through bfs_run)
    maxn = max(n for _, n, _ in graphs)
    lv = torch.empty(maxn, dtype=torch.int32, device="cuda")
    for g in range(len(pool)):
        B.bfs_run(handles[g], int(nonisolated[g][0]), lv, None, None)
    torch.cuda.synchronize()
    service = np.empty(N)
    teps = np.empty(N, np.int64)
    st = B.bfs_stats()
    for i in range(N):
        t0 = time.perf_counter()
        B.bfs_run(handles[gsel[i]], int(srcs[i]), lv, None, st)
        service[i] = time.perf_counter() - t0
        teps[i] = st.edges_scanned // 2
    capacity = 1.0 / service.mean()                       # queries per second, one at a time
    loads = [float(x) for x in str(args.serve_load).split(",")]
    base_gaps = rng.exponential(1.0, size=N)              # one Poisson stream, rescaled per load
    lines = [serve_at_load(args, B, stream, handles, graphs, gsel, srcs, service, teps, capacity, load, base_gaps,
                           t_gen) for load in loads]
    for h in handles:
        B.bfs_destroy(h)
    return lines


def serve_at_load(args, B, stream, handles, graphs, gsel, srcs, service, teps, capacity, load, base_gaps, t_gen):
    """One arrival stream at load x the one-at-a-time capacity: the server in
    real time, and first-come-first-served bfs_run from the measured service
    times."""
    N = len(gsel)
    if load > 0:
        lam = load * capacity
        arrivals = np.cumsum(base_gaps / lam)
    else:                                                 # load 0: every query at t = 0 (saturation)
        lam = float("inf")
        arrivals = np.zeros(N)
    # FCFS one at a time, from the measured service times
    done_fcfs = np.empty(N)
    t = 0.0
    for i in range(N):
        t = max(t, arrivals[i]) + service[i]
        done_fcfs[i] = t
    lat_fcfs = done_fcfs - arrivals
    # the server, in real time
    so = B.bfs_server_opts()
    so.slots = args.serve_slots
    so.local_levels = args.serve_local_levels
    so.cta_warps = args.serve_cta_warps
    so.levels_per_launch = args.serve_levels_per_launch
    srv = B.bfs_server_create(handles, so, stream.cuda_stream)
    done = {}
    # a client thread submits every query at its arrival time (a submission
    # wakes a running launch); this thread is the scheduler, polling
    import threading
    t0 = time.perf_counter()

    def client():
        for i in range(N):
            wait = arrivals[i] - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            B.bfs_server_submit(srv, int(gsel[i]), int(srcs[i]), None, None, i)

    th = threading.Thread(target=client, daemon=True)
    with ClockSampler(torch_device_index()) as clk:
        th.start()
        while len(done) < N:
            for c in B.bfs_server_poll(srv, 256):
                done[c.tag] = c
            q, r = B.bfs_server_pending(srv)
            if q == 0 and r == 0 and len(done) < N:
                time.sleep(20e-6)
        th.join()
        makespan = time.perf_counter() - t0
    B.bfs_server_destroy(srv)
    # the library stamps completions with the host's monotonic clock, the
    # clock time.perf_counter() reads on Linux: latency = done - arrival
    lat = np.array([done[i].t_done_us * 1e-6 - (t0 + arrivals[i]) for i in range(N)])
    clock_skew = float(np.median([done[i].t_submit_us * 1e-6 - (t0 + arrivals[i]) for i in range(N)]))
    status_bad = sum(int(c.status != 0) for c in done.values())
    gteps = float(teps.sum()) / makespan / 1e9
    fcfs_makespan = done_fcfs[-1] - 0.0
    line = {"metric": METRIC, "value": round(gteps, 3), "unit": "GTEPS", "n_gpus": 1, "steps": 1, "warmup": 0,
            "ms_per_step": makespan * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32", "data": "synthetic",
            "config": {"workload": "serving-pool32", "graphs": [g[0] for g in graphs], "queries": N,
                       "load": load if load > 0 else "all at t=0", "lambda_qps": lam if load > 0 else None,
                       "slots": args.serve_slots, "local_levels": args.serve_local_levels,
                       "cta_warps": args.serve_cta_warps or 16,
                       "levels_per_launch": args.serve_levels_per_launch or 64,
                       "arrivals": "Poisson, graph uniform over the pool, source uniform over non-isolated, seed 5"},
            "latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3), "p99": float(np.percentile(lat, 99) * 1e3),
                           "mean": float(lat.mean() * 1e3)},
            "fcfs_one_at_a_time": {"gteps": float(teps.sum()) / fcfs_makespan / 1e9,
                                   "p50_ms": float(np.percentile(lat_fcfs, 50) * 1e3),
                                   "p99_ms": float(np.percentile(lat_fcfs, 99) * 1e3),
                                   "capacity_qps": capacity},
            "throughput_qps": N / makespan,
            "failed": int(status_bad), "pool_build_s": round(t_gen, 1), "clocks": clk.summary(),
            "median_submit_delay_ms": clock_skew * 1e3}
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="rmat22")
    ap.add_argument("--sources", type=int, default=0, help="override the number of sources")
    ap.add_argument("--ref-sources", type=int, default=2, help="reference arm: traversals per step")
    ap.add_argument("--cpu-budget", type=float, default=12.0, help="seconds of oracle time for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--chunk-edges", type=int, default=0)
    ap.add_argument("--ctas", type=int, default=0)
    ap.add_argument("--work-insensitive", action="store_true")
    ap.add_argument("--relabel", type=int, default=0, help="bfs_opts.relabel: 0 auto, 1 always, -1 off")
    ap.add_argument("--small-level-edges", type=int, default=0,
                    help="bfs_opts.small_level_edges: 0 default, -1 off")
    ap.add_argument("--cta-warps", type=int, default=0, help="bfs_opts.cta_warps: 0 auto, 8 or 32")
    ap.add_argument("--per-phase", action="store_true", help="one launch per phase instead of the persistent loop")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--dump", default="", help="write per-traversal records of the timed steps (JSON) here")
    ap.add_argument("--levels", action="store_true", help="add the per-level statistics of the first source")
    ap.add_argument("--direction", type=int, default=0,
                    help="1: direction-optimising traversal (bottom-up levels) as the measured line")
    ap.add_argument("--autotune", action="store_true",
                    help="choose the options by the autotuner (coordinate descent on 4 of the sources)")
    ap.add_argument("--tune-cache", default="", help="JSON cache file of the autotuner")
    ap.add_argument("--do-alpha", type=int, default=0, help="bfs_opts.do_alpha (0 = 15)")
    ap.add_argument("--do-gamma", type=int, default=0, help="bfs_opts.do_gamma (0 = 2, -1 = off)")
    ap.add_argument("--do-beta", type=int, default=0, help="bfs_opts.do_beta (0 = 18)")
    ap.add_argument("--with-wi", type=int, default=1,
                    help="1 (default): add the work-insensitive arm (every warp at every level) to the line")
    ap.add_argument("--no-energy", action="store_true", help="skip the NVML energy-per-traversal loop")
    ap.add_argument("--with-do", type=int, default=1,
                    help="1 (default): add a direction-optimising run of the same sources to the top-down line")
    ap.add_argument("--batch", action="store_true",
                    help="all sources of a step in one bfs_run_batch call (64-source bitmask traversal)")
    ap.add_argument("--no-parents", action="store_true", help="levels only (batch mode)")
    ap.add_argument("--serve", action="store_true",
                    help="query server over the 32-graph pool: Poisson stream, p50/p99 latency")
    ap.add_argument("--arms", default="batch,grid,serve",
                    help="extra arms of the default R-MAT s22 line: batch (ER 2^20, 64-source bitmask), "
                         "grid (4096^2 grid, default and autotuned), serve (32-graph pool); none = only the line")
    ap.add_argument("--serve-queries", type=int, default=2000)
    ap.add_argument("--serve-load", default="0.7",
                    help="arrival rates as fractions of the one-at-a-time capacity, comma-separated; "
                         "0 = every query at t = 0 (saturation throughput)")
    ap.add_argument("--serve-slots", type=int, default=64)
    ap.add_argument("--serve-levels-per-launch", type=int, default=0,
                    help="bfs_server_opts.levels_per_launch (0 = the library default, 64)")
    ap.add_argument("--serve-cta-warps", type=int, default=0, help="bfs_server_opts.cta_warps (0 = 16)")
    ap.add_argument("--serve-local-levels", type=int, default=0,
                    help="bfs_server_opts.local_levels (0 = off)")
    args = ap.parse_args()
    w = dict(WORKLOADS[args.workload])
    if args.sources:
        w["sources"] = args.sources
    if args.impl == "reference":
        run_reference(args, w)
        return

    import torch
    from paper_2209_08764_gb300 import binding as B
    from paper_2209_08764_gb300 import replicas

    if args.serve:
        for ln in run_serve_mode(args, B, torch):
            print(json.dumps(ln), flush=True)
        return
    ws, rank, local = dist_setup()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    cpu_affinity = bind_gpu_local_cpus(torch, dev)
    B.load()

    rp, ci = make_graph(w)
    n, nnz = len(rp) - 1, len(ci)
    srcs = sources_for(w, rp, rank)
    args.cpu_affinity = cpu_affinity
    if args.batch:
        run_batch_mode(args, w, rp, ci, srcs, B, torch, dist, ws, rank, dev, replicas)
        return
    tuned, tune_info = None, None
    if args.autotune:
        from paper_2209_08764_gb300 import autotune
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        t0 = time.perf_counter()
        opts, key, info = autotune.tune(B, rp, ci, srcs[:4], cache_path=args.tune_cache or None,
                                        symmetric=True, flags=B.BFS_VALIDATE)
        tuned = autotune.resolve(opts, sms)
        tune_info = {"class": key, "chosen": opts, "tuning_s": round(time.perf_counter() - t0, 1), **info}
    direction = int(tuned.get("direction", 0)) if tuned else args.direction
    line = measure_single(args, w, rp, ci, srcs, B, torch, dist, ws, rank, dev, replicas, direction, tuned=tuned)
    if rank == 0 and tune_info:
        line["autotune"] = tune_info
    if rank == 0 and not direction and args.with_do and w["kind"] != "grid":
        # the same sources with direction-optimising levels (bottom-up where the
        # frontier is large); the headline value stays the top-down level step
        # (rank 0 alone, without collectives: the other ranks do not run these arms)
        do = measure_single(args, w, rp, ci, srcs, B, torch, None, 1, 0, dev, replicas, 1, summary=True)
        do["speedup_vs_top_down"] = round(do["value"] / line["value"], 3)
        line["direction_optimising"] = do
    if rank == 0 and not direction and args.with_wi and not args.work_insensitive:
        # the paper's comparison arm: every warp active at every level
        wi = measure_single(args, w, rp, ci, srcs, B, torch, None, 1, 0, dev, replicas, 0, summary=True,
                            tuned=dict(tuned or {}, work_insensitive=1))
        wi["time_ratio_vs_work_sensitive"] = round(wi["ms_level_step_median"] / line["ms_level_step_median"], 3)
        wi["energy_ratio_vs_work_sensitive"] = ratio_with_error(wi.get("energy"), line.get("energy"))
        line["work_insensitive"] = wi
    arms = [a for a in args.arms.split(",") if a and a != "none"]
    if rank == 0 and args.workload == "rmat22" and not direction and not tuned and not args.per_phase:
        # the rest of the metric on the same GPU, each arm on its own graph
        # (rank 0 alone: the other ranks run none of them)
        del rp, ci
        if "batch" in arms:
            line["er20_batch"] = arm_er20_batch(args, B, torch, dev, replicas, line)
        if "grid" in arms:
            line["grid4096"] = arm_grid4096(args, B, torch, dev, replicas)
        if "serve" in arms:
            line["serving"] = arm_serving(args, B, torch, line)
        rp, ci = make_graph(w)
    if rank == 0:
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(w, rp, ci, srcs, args.cpu_budget)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def arm_er20_batch(args, B, torch, dev, replicas, line):
    """Erdos-Renyi 2^20 (mean degree 16), 64 sources in one bitmask
    traversal, against the same 64 sources one at a time through bfs_run on
    the same graph."""
    w = dict(WORKLOADS["er20"])
    rp, ci = make_graph(w)
    srcs = sources_for(w, rp, 0)
    a = argparse.Namespace(**vars(args))
    a.workload, a.no_parents = "er20", False
    b = measure_batch(a, w, rp, ci, srcs, B, torch, None, 1, 0, dev, replicas)
    out = {k: b[k] for k in ("value", "unit", "steps", "ms_per_step", "config", "roofline", "clocks", "gpu_launches",
                             "sequential_gteps", "batch_speedup", "levels", "pulled_edges")}
    out["vs_rmat22_single_source_gteps"] = round(b["value"] / line["value"], 2)
    return out


GRID_TUNE_SPACE = {"cta_warps": [0, 8, 32], "small_level_edges": [0, 8192], "chunk_edges": [0, 32], "ctas": [0, -2]}


def arm_grid4096(args, B, torch, dev, replicas):
    """4096^2 grid with 1% of edges deleted: the corner (deepest source) and 7
    seeded sources, single-source S3BFS with the default options and with the
    options the autotuner picks (coordinate descent over the CTA shape, the
    small-level threshold, the grain and the grid size, on the corner
    source).  Per level
    also in SM cycles (us x the median sampled SM MHz), which takes the box's
    clock out of the comparison."""
    from paper_2209_08764_gb300 import autotune
    w = dict(WORKLOADS["grid4096"])
    rp, ci = make_graph(w)
    srcs = sources_for(w, rp, 0)
    a = argparse.Namespace(**vars(args))
    a.workload, a.steps, a.no_energy, a.levels, a.dump = "grid4096", min(args.steps, 2), True, False, ""
    out = {"config": config_of("grid4096", w, rp, ci)}
    d = measure_single(a, w, rp, ci, srcs, B, torch, None, 1, 0, dev, replicas, 0, summary=True)
    t0 = time.perf_counter()
    opts, key, info = autotune.tune(B, rp, ci, srcs[:1], symmetric=False, flags=B.BFS_VALIDATE, space=GRID_TUNE_SPACE,
                                    reps=1)
    tuned = autotune.resolve(opts, torch.cuda.get_device_properties(dev).multi_processor_count)
    tune_s = time.perf_counter() - t0
    t = measure_single(a, w, rp, ci, srcs, B, torch, None, 1, 0, dev, replicas, 0, summary=True, tuned=tuned)
    for name, r in (("default", d), ("autotuned", t)):
        mhz = (r.get("clocks") or {}).get("sm_mhz")
        out[name] = {k: r[k] for k in ("value", "unit", "ms_per_traversal_median", "ms_level_step_median",
                                       "levels_median", "us_per_level_median", "roofline", "clocks", "gpu_launches",
                                       "options")}
        out[name]["kcycles_per_level_median"] = round(r["us_per_level_median"] * mhz / 1e3, 2) if mhz else None
    out["autotune"] = {"class": key, "chosen": opts, "tuning_s": round(tune_s, 1), **info}
    out["sources"] = "corner (vertex 0) + 7 seeded non-isolated vertices"
    if not args.no_energy:
        # the paper's comparison where it matters most: thousands of small
        # levels, each on the warps (and SMs) it needs, or on every warp
        ws = energy_run(B, torch, dev, rp, ci, srcs[:1], {})
        wi = energy_run(B, torch, dev, rp, ci, srcs[:1], {"work_insensitive": 1})
        out["work_sensitive_vs_insensitive"] = {
            "source": "corner", "work_sensitive": ws, "work_insensitive": wi,
            "time_ratio_insensitive_vs_sensitive": round(wi["ms_per_traversal"] / ws["ms_per_traversal"], 3),
            "energy_ratio_insensitive_vs_sensitive": ratio_with_error(wi["energy"], ws["energy"])}
    return out


def energy_run(B, torch, dev, rp, ci, srcs, opts):
    """Time, active SMs per level and NVML energy of single-source traversals
    with the given options."""
    n = len(rp) - 1
    stream = torch.cuda.current_stream()
    o = B.bfs_opts()
    for k, v in opts.items():
        setattr(o, k, int(v))
    g = B.bfs_create_csr(n, len(ci), rp, ci, 0, o, stream.cuda_stream)
    level = torch.empty(n, dtype=torch.int32, device=dev)
    try:
        cap = 1 << 16
        buf = (ctypes.c_int32 * (cap * B.BFS_LEVEL_FIELDS))()
        st = B.bfs_stats()
        st.per_level = ctypes.cast(buf, ctypes.POINTER(ctypes.c_int32))
        st.per_level_cap = cap
        B.bfs_run(g, int(srcs[0]), level, None, None)
        B.bfs_run(g, int(srcs[0]), level, None, st)
        L = min(st.num_levels, cap)
        rows = np.frombuffer(buf, dtype=np.int32)[:L * B.BFS_LEVEL_FIELDS].reshape(L, B.BFS_LEVEL_FIELDS)
        energy = energy_per_traversal(EnergyMeter(torch, dev), lambda s: B.bfs_run(g, s, level, None, None), srcs)
        return {"options": opts, "ms_per_traversal": float(st.ms_total), "levels": int(st.num_levels),
                "active_sms": active_sms_summary(rows, sms_total(torch, dev)), "energy": energy}
    finally:
        B.bfs_destroy(g)


def arm_serving(args, B, torch, line):
    """The 32-graph pool under a Poisson stream at 0.7 of the one-at-a-time
    capacity and with every query at t = 0 (saturation), against the same
    stream served first come, first served by single-source bfs_run."""
    a = argparse.Namespace(**vars(args))
    a.serve_load = "0.7,0"
    lines = run_serve_mode(a, B, torch)
    out = {"config": dict(lines[0]["config"], load=[0.7, "all at t=0"]), "queries": a.serve_queries}
    for ln, name in zip(lines, ("load_0.7", "saturation")):
        out[name] = {"gteps": ln["value"], "latency_ms": ln["latency_ms"], "throughput_qps": ln["throughput_qps"],
                     "fcfs_one_at_a_time": ln["fcfs_one_at_a_time"], "failed": ln["failed"],
                     "clocks": ln.get("clocks")}
    out["pool_build_s"] = lines[0]["pool_build_s"]
    out["vs_rmat22_single_source_gteps"] = round(lines[1]["value"] / line["value"], 3)
    return out


def level_bytes(n, rows):
    """Algorithmic bytes of one traversal's level loop from its per-level
    records (n_l, e_l, c_l, ..., direction, work).  Top-down level: 8 per
    edge scanned (col_idx + level test) + 32 per frontier vertex + 28 per
    candidate.  Bottom-up level: 4 n (visited test of every vertex) + 8 per
    unvisited vertex (row bounds) + 8 per examined entry (col_idx + frontier
    bit test) + n / 8 (next frontier bitmap) + 36 per vertex found (level,
    parent, candidate pair and its compaction), plus 4 n + n / 8 when the
    frontier bitmap is first built from the level array."""
    total = 0.0
    visited = 0
    prev_dir = 0
    for r in rows:
        n_l, e_l, c_l, direction, work = int(r[0]), int(r[1]), int(r[2]), int(r[7]), int(r[8])
        visited += n_l
        if direction == 0:
            total += 8 * e_l + 32 * n_l + 28 * c_l
        else:
            total += 4 * n + 8 * (n - visited) + 8 * work + n / 8 + 36 * c_l
            if prev_dir == 0:
                total += 4 * n + n / 8
        prev_dir = direction
    return total


def measure_single(args, w, rp, ci, srcs, B, torch, dist, ws, rank, dev, replicas, direction, summary=False,
                   tuned=None):
    """Single-source traversals of every source, K timed steps: the bench line
    (or, with summary, its compact form for the direction-optimising run)."""
    n, nnz = len(rp) - 1, len(ci)
    deg = np.diff(rp.astype(np.int64))
    stream = torch.cuda.current_stream()
    opts = B.bfs_opts()
    opts.chunk_edges = args.chunk_edges
    opts.ctas = args.ctas
    opts.work_insensitive = 1 if args.work_insensitive else 0
    opts.persistent = -1 if args.per_phase else 0
    opts.relabel = args.relabel
    opts.small_level_edges = args.small_level_edges
    opts.cta_warps = args.cta_warps
    opts.direction = direction
    opts.do_alpha = args.do_alpha
    opts.do_gamma = args.do_gamma
    opts.do_beta = args.do_beta
    for k, v in (tuned or {}).items():
        setattr(opts, k, int(v))
    # top-down: the CSR is checked on the host (BFS_VALIDATE).  The
    # direction-optimising graph declares BFS_SYMMETRIC without that (slow)
    # host check: the generators' output is symmetric and simple, which the
    # CPU tests of graphgen pin.
    flags = B.BFS_SYMMETRIC if direction else B.BFS_VALIDATE
    opts.batch_bitmask = -1  # a batch here is single-source traversals, never one bitmask traversal
    t_create = time.perf_counter()
    g = B.bfs_create_csr(n, nnz, rp, ci, flags, opts, stream.cuda_stream)
    t_create = time.perf_counter() - t_create
    info = B.bfs_graph_info(g)
    level = torch.empty(n, dtype=torch.int32, device=dev)
    parent = torch.empty(n, dtype=torch.int32, device=dev)
    # one step = one bfs_run_batch over the sources: single-source traversals
    # queued back to back, every one writing its own level and parent arrays
    S = np.ascontiguousarray(srcs, np.int32)
    L_all = torch.empty(len(S) * n, dtype=torch.int32, device=dev)
    P_all = torch.empty(len(S) * n, dtype=torch.int32, device=dev)
    st_all = (B.bfs_stats * len(S))()

    def step(record):
        B.bfs_run_batch(g, S, len(S), L_all, P_all, st_all if record is not None else None)
        if record is None:
            return []
        return [(st.ms_level_step, st.ms_total, st.reached, st.edges_scanned, st.candidates, st.num_levels,
                 int(S[i]), st.launches, st.work_edges) for i, st in enumerate(st_all)]

    for _ in range(args.warmup):
        step(None)
    # per source: traversed edges (Graph500 count: half the degree sum of the
    # reached vertices) and the algorithmic bytes of its level loop, from one
    # untimed run with per-level records (levels, directions and work are the
    # same in every run of a source)
    cap = 1 << 16
    buf = (ctypes.c_int32 * (cap * B.BFS_LEVEL_FIELDS))()
    st2 = B.bfs_stats()
    st2.per_level = ctypes.cast(buf, ctypes.POINTER(ctypes.c_int32))
    st2.per_level_cap = cap
    teps_edges, src_bytes, first_rows, bu_levels = [], [], None, []
    for s in srcs:
        B.bfs_run(g, int(s), level, parent, st2)
        teps_edges.append(graph500_edges(deg, level.cpu().numpy(), st2))
        L = min(st2.num_levels, cap)
        rows = np.frombuffer(buf, dtype=np.int32)[:L * B.BFS_LEVEL_FIELDS].reshape(L, B.BFS_LEVEL_FIELDS).copy()
        src_bytes.append(level_bytes(n, rows) if L == st2.num_levels else np.nan)
        bu_levels.append(int((rows[:, 7] == 1).sum()))
        if first_rows is None:
            first_rows = rows
    edges_per_step = sum(teps_edges)

    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    recs = []
    with ClockSampler(dev) as clk:
        ev0.record(stream)
        # the last step records every traversal's CUDA events (its launches
        # give the per-launch durations); the others run without them, as a
        # caller that wants only throughput does (the events cost ~5 us a
        # traversal)
        for k in range(args.steps):
            recs += step(True if k == args.steps - 1 else None)
        ev1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    ms_max, total_edges = replicas.aggregate(dist, ms, edges_per_step * args.steps,
                                             torch.device("cuda", dev) if dist else None)
    gteps = total_edges / (ms_max / 1e3) / 1e9

    # roofline of the dominant kernel (the persistent level loop): algorithmic
    # bytes of each traversal's level loop / its device time
    recs = np.array(recs, dtype=np.float64)
    rec_steps = len(recs) // len(S)  # steps whose launches were timed
    ms_loop = recs[:, 0]
    bytes_loop = np.tile(np.array(src_bytes, dtype=np.float64), rec_steps)
    achieved = bytes_loop.sum() / (ms_loop.sum() / 1e3) / 1e9
    peak, peak_kind = peaks()
    traffic = profiled_traffic(args.workload, "direction_optimising" if direction else "level_loop")
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic, "peak_kind": peak_kind,
                "kernel": "k_level_loop", "algorithmic_bytes_per_launch": float(bytes_loop.mean()),
                "avg_launch_ms": float(ms_loop.mean())}
    sectors = profiled(args.workload, "l1_global_load_sectors_per_launch") if not direction else None
    if sectors and not summary and rank == 0:
        # the bound the explore actually meets: scattered loads, one L1 sector each
        peak_ld = gather_peak(torch, dev)
        ach = sectors / (ms_loop.mean() / 1e3)
        roofline["scattered_loads"] = {"bound": "l1_scattered_sectors", "achieved": ach, "peak": peak_ld,
                                       "unit": "sectors/s", "frac": round(ach / peak_ld, 4),
                                       "sectors_per_launch": sectors,
                                       "peak_kind": "measured: torch index_select of random int32"}
    hmean = len(ms_loop) / np.sum(ms_loop / 1e3 / np.tile(teps_edges, rec_steps)) / 1e9
    # launches per traversal are the same in every step
    launches = int(recs[:, 7].sum()) * args.steps // rec_steps
    energy = None
    if not args.no_energy and rank == 0:
        energy = energy_per_traversal(EnergyMeter(torch, dev), lambda s: B.bfs_run(g, s, level, parent, None), srcs)
    if summary:
        B.bfs_destroy(g)
        return {"value": round(gteps, 3), "unit": "GTEPS", "ms_per_step": ms_max / args.steps,
                "ms_level_step_median": float(np.median(ms_loop)), "roofline": roofline,
                "bottom_up_levels_median": float(np.median(bu_levels)),
                "work_edges_per_traversal": float(recs[:, 8].mean()),
                "edges_scanned_per_traversal": float(recs[:, 3].mean()),
                "gpu_launches": launches, "clocks": clk.summary(), "energy": energy,
                "options": {f: getattr(opts, f) for f, _ in opts._fields_ if getattr(opts, f)},
                "levels_median": float(np.median(recs[:, 5])),
                "us_per_level_median": float(np.median(ms_loop * 1e3 / recs[:, 5])),
                "ms_per_traversal_median": float(np.median(recs[:, 1])),
                "active_sms": active_sms_summary(first_rows, sms_total(torch, dev)),
                "create_s": round(t_create, 2)}

    # end to end through the C ABI: one bfs_run_batch call per step with
    # pinned host outputs (every traversal's level and parent reach the host
    # inside the timed region; the library overlaps each copy with the next
    # traversal)
    e2e = None
    if not args.no_e2e:
        S = np.ascontiguousarray(srcs, np.int32)
        hl = torch.empty(len(S) * n, dtype=torch.int32, pin_memory=True)
        hp = torch.empty(len(S) * n, dtype=torch.int32, pin_memory=True)
        B.bfs_run_batch(g, S[:2], min(2, len(S)), hl, hp, None)
        torch.cuda.synchronize()
        # at least 16 calls, each timed: on some boxes an occasional call runs
        # far longer than the rest, and the distribution shows it beside the mean
        calls = max(args.steps, 16)
        per_call = []
        for _ in range(calls):
            t0 = time.perf_counter()
            B.bfs_run_batch(g, S, len(S), hl, hp, None)
            per_call.append(time.perf_counter() - t0)
        te = sum(per_call)
        med = float(np.median(per_call))
        # this box's plain device -> pinned host copy rate (one traversal's
        # level array, 8 times), beside which the end-to-end number is read
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(8):
            hl[:n].copy_(L_all[:n], non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        d2h_gbs = 8 * 4 * n / (e0.elapsed_time(e1) / 1e3) / 1e9
        e2e = {"value": edges_per_step * calls / te / 1e9, "unit": "GTEPS",
               "calls": calls,
               "ms_per_call": {"mean": round(te / calls * 1e3, 2), "median": round(med * 1e3, 2),
                               "max": round(max(per_call) * 1e3, 2),
                               "slow_calls": int(sum(t > 1.2 * med for t in per_call))},
               "value_at_median_call": round(edges_per_step / med / 1e9, 3),
               "d2h_copy_gbs": round(d2h_gbs, 1), "cpu_affinity": getattr(args, "cpu_affinity", None),
               "h2d_bytes_per_step": 4 * len(srcs),
               "d2h_bytes_per_step": int(len(srcs) * (8 * n + ctypes.sizeof(ctypes.c_int64) * 8))}

    per_level = None
    if args.levels:
        rows = first_rows
        per_level = {"src": int(srcs[0]), "fields": ["n_l", "e_l", "c_l", "active_warps", "active_sms", "ns",
                                                     "ns_explore", "direction", "work"],
                     "rows": rows.tolist() if len(rows) <= 64 else rows[:64].tolist(), "levels": len(rows),
                     "ns_total": int(rows[:, 5].sum())}
    if args.dump and rank == 0:
        with open(args.dump, "w") as f:
            json.dump([{"src": int(r[6]), "ms_level_step": r[0], "ms_total": r[1], "reached": int(r[2]),
                        "edges_scanned": int(r[3]), "candidates": int(r[4]), "levels": int(r[5]),
                        "work_edges": int(r[8]), "algorithmic_bytes": float(b)}
                       for r, b in zip(recs.tolist(), bytes_loop.tolist())], f)
    line = None
    if rank == 0:
        # config: the workload alone (the reference arm prints the same);
        # method: how this arm traverses it
        config = config_of(args.workload, w, rp, ci)
        method = {"direction": "direction-optimising (alpha 15, beta 18)" if direction
                  else "top-down (S3BFS level step)",
                  "options": {f: getattr(opts, f) for f, _ in opts._fields_ if getattr(opts, f)},
                  "step": "one bfs_run_batch over the sources (single-source traversals queued back to back)"}
        line = {"metric": METRIC, "value": round(gteps, 3), "unit": "GTEPS", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
                "config": config, "method": method, "roofline": roofline,
                "clocks": clk.summary(), "gpu_launches": launches,
                "harmonic_mean_gteps_level_step": float(hmean),
                "ms_level_step_median": float(np.median(ms_loop)),
                "ms_level_step_min": float(np.min(ms_loop)), "ms_level_step_max": float(np.max(ms_loop)),
                "levels_median": float(np.median(recs[:, 5])),
                "us_per_level_median": float(np.median(ms_loop * 1e3 / recs[:, 5])),
                "ctas": info["ctas"], "warps": info["warps"],
                "active_sms": active_sms_summary(first_rows, sms_total(torch, dev))}
        if e2e:
            line["e2e"] = e2e
        line["energy"] = energy
        if per_level:
            line["per_level"] = per_level
    B.bfs_destroy(g)
    return line


if __name__ == "__main__":
    main()
