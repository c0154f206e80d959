"""Host-side logic of bench.py (CPU only): the max-over-ranks / sum-of-units
aggregation under torch.distributed (gloo, world size 2), and the JSON line of
the reference arm (the FP64 oracle on the host)."""
from __future__ import annotations

import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_WORKER = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import torch.distributed as dist
dist.init_process_group("gloo")
import bench
r = dist.get_rank()
t, u = bench.aggregate(1.0 + r, 100.0 * (r + 1))
bench.barrier()
print(json.dumps({{"rank": r, "t": t, "u": u}}), flush=True)
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_aggregate_across_two_gloo_ranks(tmp_path):
    script = tmp_path / "worker.py"
    script.write_text(_WORKER.format(root=ROOT))
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2",
                   LOCAL_RANK=str(rank))
        procs.append(subprocess.Popen([sys.executable, str(script)], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    for o in outs:
        assert o["t"] == 2.0  # slowest rank's time
        assert o["u"] == 300.0  # units of all ranks


def test_aggregate_without_process_group():
    import bench
    assert bench.aggregate(1.5, 7.0) == (1.5, 7.0)


def test_reference_arm_json(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    out = bench.run_reference(bench.main.__globals__["argparse"].Namespace(
        steps=1, warmup=3, workload=bench.DEFAULT_WORKLOAD, impl="reference"))
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in out
    assert out["impl"] == "reference" and out["value"] > 0
    assert out["e2e"]["h2d_bytes_per_step"] == 0 and out["cpu_baseline"]["kind"] == "oracle"
    json.dumps(out)
    # under torchrun only rank 0 reports
    monkeypatch.setenv("RANK", "1")
    assert bench.run_reference(bench.main.__globals__["argparse"].Namespace(
        steps=1, warmup=3, workload=bench.DEFAULT_WORKLOAD, impl="reference")) is None


def test_workloads_and_optimal_counts():
    import bench
    w = bench.workload("n28-c64-m1")
    assert w["k"] == 12867 and w["n"] == 28
    assert bench.workload("n12-c128-m1")["k"] == 50
    assert bench.workload(bench.DEFAULT_WORKLOAD)["k"] == 100


def test_gate_groups_partition_the_index_bits():
    """The group sizes the benchmark reports for each gate engine: they cover
    the n index bits exactly; CUDA cores use ceil(n/8) groups of sizes that
    differ by at most one (each group above bit 0 starts at bit 4 or higher,
    as the CUDA-core pass requires); tensor cores use 7-bit groups from bit 0
    and a shorter last one."""
    sys.path.insert(0, ROOT)
    import bench
    for n in range(1, 34):
        cc = bench.gate_groups(n, False)
        assert sum(cc) == n and len(cc) == (n + 7) // 8
        assert max(cc) - min(cc) <= 1 and max(cc) <= 8
        starts = [sum(cc[:i]) for i in range(len(cc))]
        assert all(s == 0 or s >= 4 for s in starts)
        tc = bench.gate_groups(n, True)
        assert sum(tc) == n and tc[0] == min(7, n) and all(1 <= g <= 7 for g in tc)
        assert tc == sorted(tc, reverse=True) and len(tc) == (n + 6) // 7
    assert bench.gate_groups(33, False) == [7, 7, 7, 6, 6]
    assert bench.gate_groups(33, True) == [7, 7, 7, 7, 5]
    # near-equal tensor-core groups where the greedy split leaves a short remainder
    assert bench.gate_groups(30, True) == [7, 6, 6, 6, 5]
    assert bench.gate_groups(18, True) == [7, 6, 5]
    assert bench.gate_groups(15, True) == [7, 7, 1]  # 7, 4, 4 would leave two CUDA-core groups
