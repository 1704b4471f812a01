"""Host-side pieces of bench.py (CPU): the level-loop byte model, the energy
meter's fallback without NVML, and the workload registry."""
import numpy as np

import bench


def _row(n_l, e_l, c_l, direction=0, work=None):
    # per-level record: n_l, e_l, c_l, active_warps, active_sms, ns, ns_explore, direction, work
    return [n_l, e_l, c_l, 0, 0, 0, 0, direction, e_l if work is None else work]


def test_top_down_byte_model():
    rows = [_row(1, 3, 3), _row(3, 10, 5), _row(4, 0, 0)]
    # 8 per edge scanned + 32 per frontier vertex + 28 per candidate
    assert bench.level_bytes(100, rows) == 8 * 13 + 32 * 8 + 28 * 8


def test_bottom_up_byte_model():
    n = 1000
    rows = [_row(1, 50, 40), _row(40, 900, 300, direction=1, work=700), _row(300, 2000, 10, direction=1, work=50)]
    got = bench.level_bytes(n, rows)
    td = 8 * 50 + 32 * 1 + 28 * 40
    # first bottom-up level: visited 41 after it; it also pays the bitmap build
    bu1 = 4 * n + 8 * (n - 41) + 8 * 700 + n / 8 + 36 * 300 + 4 * n + n / 8
    bu2 = 4 * n + 8 * (n - 341) + 8 * 50 + n / 8 + 36 * 10
    assert np.isclose(got, td + bu1 + bu2)


def test_energy_meter_without_nvml_is_none(monkeypatch):
    class NoNvml:
        lib = None

        def read_mj(self):
            return None
    assert bench.energy_per_traversal(NoNvml(), lambda s: None, [1, 2], seconds=0.01) is None
    assert bench.energy_per_traversal(None, lambda s: None, [1], seconds=0.01) is None


def test_workloads_are_the_documented_configurations():
    w = bench.WORKLOADS["rmat22"]
    assert (w["scale"], w["edgefactor"], w["sources"], w["seed"], w["src_seed"]) == (22, 16, 64, 1, 2)
    assert bench.WORKLOADS["grid4096"]["rows"] == bench.WORKLOADS["grid4096"]["cols"] == 4096
    assert bench.WORKLOADS["er20"]["m"] == 8 << 20


def test_cpulist_parsing():
    assert bench.parse_cpulist("0-3,8,10-11") == [0, 1, 2, 3, 8, 10, 11]
    assert bench.parse_cpulist("72-143\n") == list(range(72, 144))
    assert bench.parse_cpulist("") == []


def test_reference_arm_line():
    """bench.py --impl reference (the oracle on one host core) prints one
    JSON line with the contract's keys, on the same config as the GPU arm."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--workload",
                          "rmat16", "--steps", "1", "--warmup", "1"], capture_output=True, text=True, timeout=300,
                         cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads([x for x in out.stdout.splitlines() if x.startswith("{")][-1])
    assert line["impl"] == "reference" and line["unit"] == "GTEPS" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["steps"] == 1 and line["warmup"] == 1
    w = bench.WORKLOADS["rmat16"]
    assert line["config"]["workload"] == "rmat16" and line["config"]["sources"] == w["sources"]
    assert set(line["config"]) >= {"workload", "n", "nnz", "sources", "l2", "parallelism"}
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
