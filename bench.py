#!/usr/bin/env python3
"""Throughput benchmark of the equivalent-operator Grover iterator on GB300.

One step = one Grover search on a synthetic instance: init_uniform, k fused
iteration passes, then the measurement (success probability, norm, top-M).
The metric is amplitude-updates/s = N * k per step / time (one update = one
amplitude through one full iteration).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...   # the FP64 CPU oracle as reference arm

Prints one JSON line (rank 0).  Under torchrun every rank runs an independent
replica of the workload on its own GPU (the path is not sharded: no
collectives on the data path); value = amplitude updates of all ranks / the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# name -> (n, dtype, M, k or None for the optimal count, seed)
WORKLOADS = {
    "n33-c64-m1-k100": (33, "c64", 1, 100, 3300),
    "n28-c64-m1": (28, "c64", 1, None, 2801),
    "n28-c64-m4": (28, "c64", 4, None, 2804),
    "n28-c64-m16": (28, "c64", 16, None, 2816),
    "n28-c128-m1": (28, "c128", 1, None, 2811),
    "n28-c128-m16": (28, "c128", 16, None, 2826),
    "n26-c64-m8-k3000": (26, "c64", 8, 3000, 2608),
    "n24-c64-m1-k200": (24, "c64", 1, 200, 2401),
    "n26-c64-m1-k20": (26, "c64", 1, 20, 2621),
    "n12-c128-m1": (12, "c128", 1, None, 1201),
    "n16-c64-m1": (16, "c64", 1, None, 1601),
    "n18-c64-m1": (18, "c64", 1, None, 1801),
    "n17-c128-m1": (17, "c128", 1, None, 1711),
    "n20-c64-m1": (20, "c64", 1, None, 2001),
    "n26-c128-m1-k10": (26, "c128", 1, 10, 2631),
    "n28-c64-m1-k20": (28, "c64", 1, 20, 2801),
    "n28-c128-m1-k20": (28, "c128", 1, 20, 2811),
}
DEFAULT_WORKLOAD = "n33-c64-m1-k100"
METRIC = "amplitude-updates/s"
UNIT = "amp-updates/s"
BYTES_PER_AMP = {"c64": 8, "c128": 16}
NOMINAL_HBM_GBS = 8000.0      # GB300 HBM3e, nominal (~8 TB/s)
SMEM_BYTES_PER_CLK = 128      # shared-memory bandwidth of one SM per clock


def workload(name):
    n, dtype, m, k, seed = WORKLOADS[name]
    if k is None:
        import math
        k = int(math.floor(0.78539816339744830962 * math.sqrt((1 << n) / m)))
    return dict(name=name, n=n, dtype=dtype, M=m, k=k, seed=seed)


def describe(w):
    return (f"n={w['n']} {'complex64' if w['dtype'] == 'c64' else 'complex128'}, M={w['M']} seeded marked "
            f"indices, uniform init, {w['k']} iterations + init + measure per step")


def config_of(w, n_gpus, path="auto"):
    state_bytes = (1 << w["n"]) * BYTES_PER_AMP[w["dtype"]]
    l2 = (f"inputs larger than L2 ({state_bytes / 2**30:.1f} GiB state, 129 MB L2)" if state_bytes > 129e6 else
          f"state of {state_bytes / 2**20:.2f} MiB stays on chip / in L2 by design (small-state workload)")
    return {"workload": describe(w), "name": w["name"], "n": w["n"], "state_dtype": w["dtype"], "M": w["M"],
            "k": w["k"], "seed": w["seed"], "state_bytes": state_bytes, "l2": l2, "path": path,
            "parallelism": f"replicas x{n_gpus}"}


# ---- distributed plumbing (host-side barrier and max over ranks only) -------------------
def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def aggregate(elapsed_s: float, units: float, backend_device="cpu"):
    """(max elapsed over ranks, sum of units over ranks); identity without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return elapsed_s, units
    t = torch.tensor([elapsed_s], dtype=torch.float64, device=backend_device)
    u = torch.tensor([units], dtype=torch.float64, device=backend_device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


# ---- clocks -----------------------------------------------------------------------------------------
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={CLOCK_FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


# ---- roofline inputs ----------------------------------------------------------------------------------
def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0}, "fallback"


def kernel_source_hash():
    """sha256[:16] of k_stream.cu's code with comments and blank space
    removed, so that a comment edit does not invalidate recorded counters."""
    p = os.path.join(ROOT, "paper_2005_04635_gb300", "csrc", "k_stream.cu")
    text = open(p).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    text = re.sub(r"\s+", " ", text).strip()
    return hashlib.sha256(text.encode()).hexdigest()[:16]


def pass_kernel_name(dtype, N):
    """The iteration kernel grover_iterate runs by default (grover.h,
    GROVER_OPT_STAGED_PASS): the staged pass for complex64 states larger than
    half the L2, else the per-thread pass."""
    import torch
    l2 = torch.cuda.get_device_properties(0).L2_cache_size
    if dtype == "c64" and N * BYTES_PER_AMP[dtype] > l2 // 2:
        return ("k_pass_bulk (fused oracle + inversion about the mean + next-mean partial sums, "
                "16 KiB chunks staged through shared memory by bulk copies)")
    return "k_pass (fused oracle + inversion about the mean + next-mean partial sums)"


def recorded_traffic(w):
    """DRAM bytes per launch of the iteration pass from a committed ncu summary,
    scaled to this workload's N; None if no summary matches the current source."""
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return None
    src = kernel_source_hash()
    for fn in sorted(os.listdir(pdir)):
        if not fn.endswith(".md"):
            continue
        text = open(os.path.join(pdir, fn)).read()
        mh = re.search(r"k_stream\.cu sha256\[:16\]:\s*`?([0-9a-f]{16})", text)
        mt = re.search(r"traffic_bytes_per_amp_" + w["dtype"] + r":\s*([0-9.]+)", text)
        if mh and mt and mh.group(1) == src:
            return float(mt.group(1)) * (1 << w["n"])
    return None


def hbm_roofline(bytes_per_launch, launch_s, kernel, peaks, peak_src, traffic=None):
    """Roofline record of an HBM-bound kernel: algorithmic bytes per launch over
    its average launch time, against the measured copy bandwidth and the
    nominal HBM bandwidth."""
    achieved = bytes_per_launch / launch_s / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "peak_nominal": NOMINAL_HBM_GBS,
            "frac_nominal": achieved / NOMINAL_HBM_GBS, "traffic": traffic, "kernel": kernel,
            "algorithmic_bytes_per_launch": bytes_per_launch, "avg_launch_ms": launch_s * 1e3,
            "peak_source": f"{peak_src} hbm_gbs"}


def smem_peak_gbs(sm_count, sm_mhz):
    """Shared-memory bandwidth of all SMs: 128 bytes per clock per SM."""
    return sm_count * SMEM_BYTES_PER_CLK * sm_mhz * 1e6 / 1e9


def smem_roofline(bytes_per_iter, iter_s, kernel, sm_count, sm_mhz, note):
    achieved = bytes_per_iter / iter_s / 1e9
    peak = smem_peak_gbs(sm_count, sm_mhz)
    return {"bound": "smem", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": None, "kernel": kernel, "algorithmic_bytes_per_launch": None,
            "algorithmic_bytes_per_iteration": bytes_per_iter, "iteration_us": iter_s * 1e6,
            "peak_source": f"{sm_count} SMs x {SMEM_BYTES_PER_CLK} B/clock x {sm_mhz:.0f} MHz (sampled SM clock)",
            "note": note}


def p_success_closed_form(n, m, k):
    """sin^2((2k+1) theta), sin theta = sqrt(M/N): the textbook rotation picture
    of the Grover iteration for a uniform start."""
    import math
    theta = math.asin(math.sqrt(m / (1 << n)))
    return math.sin((2 * k + 1) * theta) ** 2


def resident_kernel(n, dtype):
    """The on-chip iterator grover_iterate picks (grover.h, GROVER_OPT_RESIDENT)."""
    return "k_resident_cluster" if n <= (12 if dtype == "c64" else 11) else "k_resident_grid"


# ---- CPU baseline: the FP64 oracle on the host cores --------------------------------------------------
def cpu_model():
    """The host CPU's model name as lscpu reports it (else the platform string)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


_CPU_WORKER = r"""
import sys, time, json
sys.path.insert(0, {root!r})
import oracle
from paper_2005_04635_gb300 import inputs
n, seed, seconds = {n}, {seed}, {seconds}
marked = inputs.marked_indices(n, 1, seed)
psi = oracle.init_uniform(n)
t0 = time.perf_counter()
oracle.grover_operator(psi, n, marked, 1)
t1 = time.perf_counter()
iters = max(1, int(seconds / max(t1 - t0, 1e-6)) - 1)
t2 = time.perf_counter()
oracle.grover_operator(psi, n, marked, iters)
t3 = time.perf_counter()
print(json.dumps({{"updates": (1 << n) * (iters + 1), "seconds": (t1 - t0) + (t3 - t2)}}), flush=True)
"""


def _oracle_processes(count, n, seconds, seed):
    """`count` independent processes, each running the plain FP64 oracle on its
    own seeded instance; returns [(updates, seconds)] per process."""
    procs = [subprocess.Popen([sys.executable, "-c", _CPU_WORKER.format(root=ROOT, n=n, seed=seed + i,
                                                                         seconds=seconds)],
                              stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True) for i in range(count)]
    res = []
    for p in procs:
        out, err = p.communicate(timeout=600)
        if p.returncode != 0:
            raise RuntimeError(f"oracle worker failed: {err.strip()[-300:]}")
        r = json.loads(out.strip().splitlines()[-1])
        res.append((r["updates"], r["seconds"]))
    return res


def cpu_baseline(seconds: float = 10.0, n: int = 24, seed: int = 2401):
    """The plain FP64 oracle (operator form, one thread per process) on a bounded
    sample: one process (the paper's single-thread setup), then one process per
    host core on independent instances at once (sum of their throughputs).
    Processes are started fresh (no fork of this CUDA process)."""
    one = _oracle_processes(1, n, seconds, seed)
    value1 = one[0][0] / one[0][1]
    cores = host_cores()
    many = _oracle_processes(cores, n, seconds, seed + 100)
    value_all = sum(u / t for u, t in many)
    return {"value": value1, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"n={n} (2^{n} complex128 amplitudes), M=1, uniform init, {one[0][0] >> n} iterations of the "
                      f"FP64 operator oracle (plain C, one thread), {one[0][1]:.1f} s",
            "cpu_model": cpu_model(), "host_cores": cores,
            "all_cores": {"value": value_all, "unit": UNIT, "cores": cores, "processes": cores,
                          "sample": f"{cores} processes at once, each the one-thread oracle on its own seeded n={n} "
                                    f"instance for about {seconds:.0f} s; value = sum of their throughputs"}}


# ---- our arm -------------------------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_2005_04635_gb300 import binding, inputs
    binding.lib()
    w = workload(args.workload)
    n, dtype, M, k = w["n"], w["dtype"], w["M"], w["k"]
    N = 1 << n
    marked = inputs.marked_indices(n, M, w["seed"])
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    st = binding.State(n, dtype, device=dev, stream=stream)
    st.set_resident({"auto": -1, "pass": 0, "resident": 1}[args.path])
    mk = binding.Marked(n, marked)

    ev_it = []

    def step(record=False):
        st.init_uniform()
        if record:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
        st.iterate(mk, k)
        if record:
            b.record(stream)
            ev_it.append((a, b))
        ps, nrm = st.success_prob(mk)
        idx, p = st.measure_topm(min(M, 16))
        return ps, nrm, idx

    for _ in range(args.warmup):
        step()
    st.sync()
    barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        ps, nrm, idx = step(record=True)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier()
    elapsed = e0.elapsed_time(e1) / 1e3
    st.sync()
    units = float(N) * k * args.steps
    t_max, units_all = aggregate(elapsed, units, backend_device=dev)
    value = units_all / t_max
    iter_ms = sum(a.elapsed_time(b) for a, b in ev_it)
    pass_s = iter_ms / 1e3 / (args.steps * k)

    # end-to-end through the C ABI: host marked list (pinned) in, host results out
    pinned = torch.empty(M, dtype=torch.int64, pin_memory=True)
    pinned.numpy()[:] = marked.astype(np.int64)
    host_idx = pinned.numpy().view(np.uint64)
    torch.cuda.synchronize()
    barrier()
    e2e_steps = max(1, min(args.steps, 5))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        mk2 = binding.Marked(n, host_idx)
        st.init_uniform()
        st.iterate(mk2, k)
        st.success_prob(mk2)
        st.measure_topm(min(M, 16))
        mk2.close()
    torch.cuda.synchronize()
    e2e_elapsed = time.perf_counter() - t0
    e2e_t, e2e_units = aggregate(e2e_elapsed, float(N) * k * e2e_steps, backend_device=dev)

    # the conventional circuit on the same state, for the speedup of the
    # equivalent operator over it (a few iterations; not part of `value`):
    # every engine that runs this state
    gate = None
    if args.gate_iters > 0:
        gate = {"iterations_timed": args.gate_iters, "unit": UNIT}
        engines = ([("tensor_cores", 1), ("cuda_cores", 0), ("default", -1)] if (dtype == "c64" and n >= 13)
                   else [("cuda_cores", 0)])
        for name, eng in engines:
            st.set_gate_engine(eng)
            st.init_uniform()
            st.iterate_gate(mk, 1)  # warm-up
            torch.cuda.synchronize()
            g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            g0.record(stream)
            st.iterate_gate(mk, args.gate_iters)
            g1.record(stream)
            torch.cuda.synchronize()
            st.sync()
            gate_s = g0.elapsed_time(g1) / 1e3 / args.gate_iters
            groups, on_tc = gate_engine_groups(n, eng) if dtype == "c64" else (gate_groups(n, False), False)
            passes = 2 * len(groups)
            gate[name] = {"iteration_ms": gate_s * 1e3, "value": N / gate_s, "passes_per_iteration": passes,
                          "group_bits": groups,
                          "tensor_core_groups": [kb for i, kb in enumerate(groups)
                                                 if on_tc and tc_pass_supported(n, sum(groups[:i]), kb)],
                          "hbm_gbs": passes * 2 * BYTES_PER_AMP[dtype] * N / gate_s / 1e9,
                          "hbm_frac": passes * 2 * BYTES_PER_AMP[dtype] * N / gate_s / 1e9 / measured_peaks()[0]["hbm_gbs"],
                          "operator_speedup": gate_s / pass_s}
        st.set_gate_engine(-1)
        # gate by gate (one pass per single-qubit gate, Fig. oracle1 oracle):
        # the paper's (f_o + f_c + 2n)-gate cost model; one iteration
        st.init_uniform()
        st.iterate_circuit(mk, 1)  # warm-up
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        gates, passes = st.iterate_circuit(mk, 1)
        g1.record(stream)
        torch.cuda.synchronize()
        st.sync()
        gate_s = g0.elapsed_time(g1) / 1e3
        gate["gate_by_gate"] = {"iteration_ms": gate_s * 1e3, "value": N / gate_s, "gates_per_iteration": gates,
                                "passes_per_iteration": passes,
                                "hbm_gbs": passes * 2 * BYTES_PER_AMP[dtype] * N / gate_s / 1e9,
                                "operator_speedup": gate_s / pass_s}

    n28 = None
    if args.n28 and args.workload == DEFAULT_WORKLOAD:
        n28 = n28_records(binding, inputs, stream)

    if rank != 0:
        return None
    # the library's choice of a persistent on-chip iterator (grover.h,
    # GROVER_OPT_RESIDENT: cluster or grid kernel up to n = 22 / 21)
    resident = args.path in ("auto", "resident") and n <= (22 if dtype == "c64" else 21)
    peaks, peak_src = measured_peaks()
    if resident:
        sm_count = torch.cuda.get_device_properties(0).multi_processor_count
        sm_mhz = clk.get("sm_mhz") or peaks.get("sm_max_mhz") or 2070.0
        roofline = smem_roofline(
            2 * BYTES_PER_AMP[dtype] * N, pass_s, resident_kernel(n, dtype), sm_count, sm_mhz,
            "the state stays in shared memory for all k iterations (one launch); per iteration every amplitude is "
            "read and written once there; the iteration time is set by the latency of the per-iteration exchange "
            "of exact partial sums, not by this bandwidth")
    else:
        roofline = hbm_roofline(BYTES_PER_AMP[dtype] * 2 * N, pass_s, pass_kernel_name(dtype, N), peaks, peak_src,
                                recorded_traffic(w))
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if dtype == "c64" else "f64",
        "data": "synthetic (seeded marked indices, uniform initial state)",
        "config": config_of(w, world, args.path),
        "roofline": roofline,
        "iteration_us": pass_s * 1e6,
        "e2e": {"value": e2e_units / e2e_t, "unit": UNIT, "h2d_bytes_per_step": 8 * M,
                "d2h_bytes_per_step": 16 * min(M, 16) + 16, "steps": e2e_steps},
        "gpu_launches": args.steps * ((1 if resident else k + 1) + 4),
        "clocks": clk,
        "result_check": {"p_success": ps, "p_success_closed_form": p_success_closed_form(n, M, k), "norm": nrm,
                         "top": [int(x) for x in idx]},
        "gate_path": gate,
    }
    if n28 is not None:
        out["n28"] = n28
    if not args.no_cpu_baseline:
        cb = cpu_baseline()
        cb["gpu_over_cpu"] = {"one_core": value / cb["value"], "all_cores": value / cb["all_cores"]["value"],
                              "note": "GPU complex64 value over the FP64 oracle's amplitude-updates/s (complex128)"}
        out["cpu_baseline"] = cb
    return out


# n = 28 half of the metric: full optimal k, one search each, outside the timed
# region of `value`
N28_WORKLOADS = ("n28-c64-m1", "n28-c64-m4", "n28-c64-m16", "n28-c128-m1")


def n28_records(binding, inputs, stream):
    """One full search per n = 28 workload (k = floor(pi/4 sqrt(N/M))): the
    iteration pass's time per launch from CUDA events on the launching stream,
    its HBM roofline, and P_success against the closed form."""
    import torch
    peaks, peak_src = measured_peaks()
    recs = []
    for name in N28_WORKLOADS:
        w = workload(name)
        n, dtype, M, k = w["n"], w["dtype"], w["M"], w["k"]
        N = 1 << n
        marked = inputs.marked_indices(n, M, w["seed"])
        mk = binding.Marked(n, marked)
        st = binding.State(n, dtype, stream=stream)
        st.init_uniform()
        st.iterate(mk, 3)  # warm-up
        st.init_uniform()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st.iterate(mk, k)
        b.record(stream)
        ps, nrm = st.success_prob(mk)
        idx, _ = st.measure_topm(min(M, 16))
        st.sync()
        it_s = a.elapsed_time(b) / 1e3 / k
        p_cf = p_success_closed_form(n, M, k)
        tol = 1e-4 if dtype == "c64" else 1e-11
        recs.append({
            "workload": describe(w), "name": name, "n": n, "state_dtype": dtype, "M": M, "k": k, "seed": w["seed"],
            "iteration_us": it_s * 1e6, "value": N / it_s, "unit": UNIT,
            "roofline": hbm_roofline(2 * BYTES_PER_AMP[dtype] * N, it_s, pass_kernel_name(dtype, N), peaks, peak_src,
                                     recorded_traffic(w)),
            "p_success": ps, "p_success_closed_form": p_cf, "p_success_err": abs(ps - p_cf),
            "p_success_tolerance": tol, "p_success_ok": abs(ps - p_cf) <= tol,
            "norm_err": abs(1.0 - nrm), "top_m_is_marked": sorted(int(x) for x in idx) == sorted(int(x) for x in marked)})
        del st, mk
        torch.cuda.empty_cache()
    return recs


def tc_pass_supported(n, lo, kb):
    """The groups the tensor-core pass takes (the others run on CUDA cores)."""
    if lo == 0:
        return kb == 7 and n >= 13
    return 5 <= kb <= 7 and lo >= 13 - kb and lo + kb <= n


GATE_TC_AUTO_MIN_QUBITS = 26


def gate_engine_groups(n, engine):
    """(group sizes, tensor cores used) of grover_iterate_gate for a complex64
    state (grover.h, GROVER_OPT_GATE_ENGINE): 0 CUDA cores, 1 tensor cores,
    -1 the default (CUDA cores below n = 26, else the plan with fewer groups,
    ties to the 7-bit one, tensor cores on every group they take)."""
    if engine == 1:
        return gate_groups(n, True), True
    if engine == 0 or n < GATE_TC_AUTO_MIN_QUBITS:
        return gate_groups(n, False), False
    t, c = gate_groups(n, True), gate_groups(n, False)
    return (t if len(t) <= len(c) else c), True


def gate_groups(n, tensor_cores):
    """Index-bit group sizes of one H^{(x)n} in grover_iterate_gate: tensor
    cores take 7 bits from bit 0 and the rest in 7-bit groups, or in near-equal
    groups where that leaves fewer groups they cannot take; CUDA cores use
    ceil(n / 8) groups of balanced sizes."""
    if tensor_cores:
        greedy = [7] * (n // 7) + ([n % 7] if n % 7 else [])
        parts = len(greedy) - 1
        if n < 13 or parts < 1:
            return greedy
        rest = n - 7
        bal = [7] + [rest // parts + (1 if j < rest % parts else 0) for j in range(parts)]

        def fallbacks(gs):
            return sum(not tc_pass_supported(n, sum(gs[:i]), k) for i, k in enumerate(gs))
        return bal if fallbacks(bal) < fallbacks(greedy) else greedy
    g = (n + 7) // 8
    return [n // g + (1 if i < n % g else 0) for i in range(g)]


# ---- batched: 4096 independent searches in one persistent launch --------------------------------------
def batched_instances(count=4096, seed=4096):
    """n ~ U[8, 20], M ~ U[1, 8] seeded marked indices, k = floor(pi/4 sqrt(N/M))."""
    import math
    from paper_2005_04635_gb300 import inputs
    g = inputs.rng(seed)
    ns = [int(x) for x in g.integers(8, 21, count)]
    ms = [int(x) for x in g.integers(1, 9, count)]
    marks = [inputs.marked_indices(n, m, seed * 10007 + i) for i, (n, m) in enumerate(zip(ns, ms))]
    ks = [int(math.floor(0.78539816339744830962 * math.sqrt((1 << n) / m))) for n, m in zip(ns, ms)]
    return ns, ks, marks


def run_batched(args):
    import math

    import numpy as np
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_2005_04635_gb300 import binding
    binding.lib()
    ns, ks, marks = batched_instances()
    stream = torch.cuda.current_stream()
    b = binding.Batch(ns, ks, marks, stream=stream)
    threads, onchip = b.tune()
    pack_size, pack_min = b.packing()
    for _ in range(args.warmup):
        b.run()
    b.success()
    barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        b.run()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    p = b.success()
    elapsed = e0.elapsed_time(e1) / 1e3
    units = float(sum((1 << n) * k for n, k in zip(ns, ks))) * args.steps
    t_max, units_all = aggregate(elapsed, units, backend_device=torch.device("cuda", torch.cuda.current_device()))
    # end to end: instance tables from the host, results back to the host
    t0 = time.perf_counter()
    e2e_steps = max(1, min(args.steps, 3))
    for _ in range(e2e_steps):
        b2 = binding.Batch(ns, ks, marks, stream=stream)
        b2.run()
        b2.success()
        b2.close()
    torch.cuda.synchronize()
    e2e_t = time.perf_counter() - t0
    if rank != 0:
        return None
    # closed-form check of every instance's success probability
    worst = 0.0
    for n, k, mk, pi in zip(ns, ks, marks, p):
        theta = math.atan2(math.sqrt(len(mk)), math.sqrt((1 << n) - len(mk)))
        worst = max(worst, abs(pi - math.sin((2 * k + 1) * theta) ** 2))
    # HBM bytes: streamed instances read + write every iteration; on-chip ones
    # (one CTA, or a group of CTAs) are written once at the end
    onchip_amps = 2 * onchip
    sm_count0 = torch.cuda.get_device_properties(0).multi_processor_count

    def on_chip(n):
        return (1 << n) <= onchip_amps or (pack_size == 2 and n >= pack_min and (1 << n) * 8 <= sm_count0 * 225 * 1024)
    hbm = sum(8 * (1 << n) if on_chip(n) else 16 * (1 << n) * k + 8 * (1 << n) for n, k in zip(ns, ks))
    peaks, peak_src = measured_peaks()
    achieved = hbm * args.steps / t_max / 1e9
    h2d = 4 * len(ns) + 8 * len(ns) + 8 * sum(len(x) for x in marks) + 8 * (len(ns) + 1)
    # the classes of instances, each timed alone (same kernel choices) against
    # its own bound: one CTA per instance in shared memory (n up to the tuned
    # on-chip size), groups of CTAs holding the state in shared memory (the
    # packing chosen by the tuner), and the rest streamed through L2 / HBM
    sm_count = torch.cuda.get_device_properties(0).multi_processor_count
    sm_mhz = clk.get("sm_mhz") or peaks.get("sm_max_mhz") or 2070.0
    group_ok = lambda n: n >= pack_min and (1 << n) * 8 <= sm_count * 225 * 1024
    cls_of = {}
    for i, n in enumerate(ns):
        if (1 << n) <= onchip_amps:
            cls_of[i] = "onchip"
        elif pack_size == 2 and group_ok(n):
            cls_of[i] = "groups"
        elif pack_size == 16 and n >= max(pack_min, 17):
            cls_of[i] = "clusters"
        else:
            cls_of[i] = "streamed"
    parts = {}
    for part in ("onchip", "groups", "clusters", "streamed"):
        sub = [i for i in range(len(ns)) if cls_of[i] == part]
        if not sub:
            continue
        sn, sk, sm_ = [ns[i] for i in sub], [ks[i] for i in sub], [marks[i] for i in sub]
        b3 = binding.Batch(sn, sk, sm_, stream=stream)
        th3, oc3 = b3.tune()
        b3.set_packing(pack_size, pack_min)
        for _ in range(2):
            b3.run()
        t3 = _timed_events(b3.run, max(1, min(args.steps, 5)), stream)
        b3.close()
        units3 = float(sum((1 << n) * k for n, k in zip(sn, sk)))
        rec = {"instances": len(sub), "n_range": [min(sn), max(sn)], "ms_per_launch": t3 * 1e3,
               "value": units3 / t3, "unit": UNIT, "tuned_one_cta": {"threads": th3, "onchip_vecs": oc3}}
        if part in ("onchip", "groups"):
            rec["roofline"] = smem_roofline(
                16.0 * units3, t3,
                "k_batch (instances in shared memory)" if part == "onchip" else
                f"k_batch_group (groups of CTAs, n >= {pack_min})", sm_count, sm_mhz,
                "the states stay in shared memory for all k_i iterations; bytes = 16 per amplitude-update (read + "
                "write in shared memory), the whole class per launch" +
                ("; per iteration the CTAs of a group exchange exact partial sums through global memory, which "
                 "bounds the iteration" if part == "groups" else ""))
            rec["roofline"]["algorithmic_bytes_per_iteration"] = None
            rec["roofline"]["iteration_us"] = None
            rec["roofline"]["algorithmic_bytes_per_launch"] = 16.0 * units3
            rec["hbm_equivalent_gbs"] = 16.0 * units3 / t3 / 1e9
        else:
            rec["roofline"] = hbm_roofline(
                sum(16 * (1 << n) * k + 8 * (1 << n) for n, k in zip(sn, sk)), t3,
                "k_batch (streamed instances)" if part == "streamed" else f"k_batch_cluster (n >= {pack_min})",
                peaks, peak_src)
        parts[part] = rec
    return {
        "metric": METRIC, "value": units_all / t_max, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (4096 seeded instances, uniform initial states)",
        "config": {"workload": "batched: 4096 independent searches, n ~ U[8,20], M ~ U[1,8], k_i optimal, "
                               "complex64, one persistent CUDA-graph launch per step", "name": "batched-4096",
                   "instances": len(ns), "amp_updates_per_step": units / args.steps,
                   "tuned": {"threads": threads, "onchip_vecs": onchip,
                             "packing": {1: "one CTA per instance", 2: "groups of CTAs in shared memory",
                                         16: "clusters of 16 CTAs"}.get(pack_size, str(pack_size)),
                             "packing_min_qubits": pack_min if pack_size > 1 else None},
                   "l2": "per-step traffic 16 B x N x k of the streamed instances (> L2 in total)",
                   "parallelism": f"replicas x{world}"},
        "roofline": dict(hbm_roofline(hbm, t_max / args.steps, "k_batch + k_batch_group / k_batch_cluster",
                                      peaks, peak_src),
                         note="mixed graph: instances held in shared memory (one CTA, or a group of CTAs) move no "
                              "HBM bytes per iteration; the per-class records in `parts` give each class against its "
                              "own bound"),
        "parts": parts,
        "e2e": {"value": float(sum((1 << n) * k for n, k in zip(ns, ks))) * e2e_steps / e2e_t, "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 8 * len(ns), "steps": e2e_steps},
        "gpu_launches": args.steps, "clocks": clk,
        "result_check": {"max_abs_p_success_error_vs_closed_form": worst},
    }


# ---- precision study: FP32 storage, mean accumulation modes vs the FP64 oracle ------------------------
PRECISION_MODES = ("fp32", "kahan", "fp64", "default", "exact")


def run_precision_study(args):
    """n=26 i.i.d. complex Gaussian start (unit norm), M=8, 3000 iterations,
    complex64 storage under every mean accumulation mode, complex128 for
    comparison; errors against the FP64 oracle's closed form for an arbitrary
    start (the rotation of the marked / unmarked means, O(N) for any k).  The
    mean of a Gaussian start is tiny, so the same runs from the uniform start
    (where the mean is ~1/sqrt(N) and the run passes the optimum, k = 2274) show
    how the accumulation modes differ."""
    import numpy as np
    import torch

    import oracle
    from paper_2005_04635_gb300 import binding, inputs
    torch.cuda.set_device(0)
    binding.lib()
    n, m, k, seed = 26, 8, 3000, 2608
    marked = inputs.marked_indices(n, m, seed)
    psi = inputs.gaussian_state(n, seed + 1)
    psi32 = psi.astype(np.complex64)
    ref = oracle.closed_form_general(psi32.astype(np.complex128), n, marked, k)
    ref128 = oracle.closed_form_general(psi.copy(), n, marked, k)
    p_ref = oracle.success_prob(ref, n, marked)
    mk = binding.Marked(n, marked)
    rows = []
    a_m, a_u = oracle.closed_form_uniform(n, m, k)
    mask = np.zeros(1 << n, dtype=bool)
    mask[marked.astype(np.int64)] = True
    for start in ("gaussian", "uniform"):
        for dtype, mode in [("c64", md) for md in PRECISION_MODES] + [("c128", "default")]:
            st = binding.State(n, dtype)
            if mode != "default":
                st.set_accum(mode)
            st.set_resident(0)
            if start == "gaussian":
                st.init_state(psi32 if dtype == "c64" else psi)
            else:
                st.init_uniform()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            st.iterate(mk, k)
            e1.record()
            ps, nrm = st.success_prob(mk)
            got = st.amps.cpu().numpy().astype(np.complex128)
            if start == "gaussian":
                r = ref if dtype == "c64" else ref128
                pr = oracle.success_prob(r, n, marked)
                err = float(np.max(np.abs(got - r)))
            else:
                pr = m * a_m * a_m
                err = float(max(np.max(np.abs(got[mask] - a_m)), np.max(np.abs(got[~mask] - a_u))))
            rows.append({"start": start, "state": dtype, "accumulation": mode, "max_abs_err": err,
                         "p_success": ps, "p_success_err": abs(ps - pr), "norm_err": abs(1.0 - nrm),
                         "iteration_us": e0.elapsed_time(e1) * 1e3 / k,
                         "value": (1 << n) * k / (e0.elapsed_time(e1) / 1e3)})
            del st, got
            torch.cuda.empty_cache()
    return {"study": "precision", "workload": f"n={n}, M={m} (seed {seed}), {k} iterations; complex Gaussian "
            f"start (seed {seed + 1}) as specified, and the uniform start for contrast",
            "p_success_fp64": {"gaussian": p_ref, "uniform": m * a_m * a_m},
            # worst-case 2-norm of the complex64 error vector (default accumulation,
            # the streaming pass these runs take): per iteration 8u + 64u^2 (FP32
            # pairwise 8-amplitude tile sums of the mean, two roundings per stored
            # amplitude), u = 2^-24, plus u for the start
            "bound_error_norm_c64_default": (1 + 8 * 2.0 ** -24 + 64 * 2.0 ** -48) ** k * (1 + 2.0 ** -24) - 1,
            "rows": rows}


def run_phase_study(args):
    """Generalised phase iterator with its adjoint: n=20, M=3, K=32, phases
    U(0, 2 pi), uniform start, loss -log P.  Gradient errors against FP64
    central differences (h=1e-6) of the exact two-amplitude model and against
    central differences (h=1e-4) of the GPU loss; 200 Adam steps through the
    torch.autograd.Function; forward / backward times per iteration next to the
    plain iterator at n=20 (L2-resident) and n=28 (HBM-bound)."""
    import math

    import numpy as np
    import torch

    import oracle
    from paper_2005_04635_gb300 import binding, inputs
    from paper_2005_04635_gb300.autograd import phase_search_loss
    torch.cuda.set_device(0)
    binding.lib()
    n, m, K, seed = 20, 3, 32, 750
    marked = inputs.marked_indices(n, m, seed)
    phi0, vphi0 = inputs.uniform_phases(K, seed + 1)
    dev = lambda a: torch.as_tensor(np.asarray(a, dtype=np.float64), device="cuda").contiguous()
    mk = binding.Marked(n, marked)
    st = binding.State(n, "c64")
    stats = torch.zeros(2, dtype=torch.float64, device="cuda")
    lam = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    gp = torch.empty(K, dtype=torch.float64, device="cuda")
    gv = torch.empty(K, dtype=torch.float64, device="cuda")
    st.init_uniform()
    st.phase_forward(mk, dev(phi0), dev(vphi0), stats)
    st.phase_backward(mk, dev(phi0), dev(vphi0), lam, gp, gv)
    torch.cuda.synchronize()
    L_ref = oracle.phase_reduced(n, m, phi0, vphi0)[0]
    L_gpu = float(stats[1].item())
    fp, fv = oracle.phase_grad_fd(lambda a, b: oracle.phase_reduced(n, m, a, b)[0], phi0, vphi0, h=1e-6)
    scale = float(max(np.max(np.abs(fp)), np.max(np.abs(fv))))
    g_phi, g_vphi = gp.cpu().numpy(), gv.cpu().numpy()
    err_fp64 = float(max(np.max(np.abs(g_phi - fp)), np.max(np.abs(g_vphi - fv))))

    def gpu_loss(a, b):
        st.init_uniform()
        st.phase_forward(mk, dev(a), dev(b), stats)
        torch.cuda.synchronize()
        return float(stats[1].item())

    h, fd_err = 1e-4, 0.0
    for t in range(K):
        for arr, g in ((phi0, g_phi), (vphi0, g_vphi)):
            up, dn = arr.copy(), arr.copy()
            up[t] += h
            dn[t] -= h
            d = ((gpu_loss(up, vphi0) - gpu_loss(dn, vphi0)) if arr is phi0 else
                 (gpu_loss(phi0, up) - gpu_loss(phi0, dn))) / (2 * h)
            fd_err = max(fd_err, abs(d - g[t]))

    # 200 Adam steps, after one untimed step on copies (the optimizer's own
    # kernels load on first use)
    wp = dev(phi0).requires_grad_(True)
    wv = dev(vphi0).requires_grad_(True)
    wopt = torch.optim.Adam([wp, wv], lr=0.05)
    wopt.zero_grad()
    phase_search_loss(wp, wv, st, mk).backward()
    wopt.step()
    phi = dev(phi0).requires_grad_(True)
    vphi = dev(vphi0).requires_grad_(True)
    opt = torch.optim.Adam([phi, vphi], lr=0.05)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(200):
        opt.zero_grad()
        loss = phase_search_loss(phi, vphi, st, mk)
        loss.backward()
        opt.step()
    torch.cuda.synchronize()
    adam_s = time.perf_counter() - t0
    final = float(phase_search_loss(phi.detach(), vphi.detach(), st, mk).item())
    final_ref = oracle.phase_reduced(n, m, phi.detach().cpu().numpy(), vphi.detach().cpu().numpy())[0]
    theta = math.asin(math.sqrt(m / (1 << n)))

    # per-iteration times: forward, backward, plain iterator (pass path)
    def timed(fn, reps=5):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / reps

    peaks, peak_src = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    sizes = []
    for nn in (20, 28):
        mk2 = binding.Marked(nn, inputs.marked_indices(nn, m, seed + nn))
        s2 = binding.State(nn, "c64")
        lam2 = torch.empty(1 << nn, dtype=torch.complex64, device="cuda")
        p_, v_ = dev(phi0), dev(vphi0)
        s2.init_uniform()
        fwd = timed(lambda: s2.phase_forward(mk2, p_, v_, None))
        bwd = timed(lambda: (s2.phase_forward(mk2, p_, v_, None),
                             s2.phase_backward(mk2, p_, v_, lam2, gp, gv))) - fwd
        s2.set_resident(0)
        plain = timed(lambda: s2.iterate(mk2, K))
        N = 1 << nn
        row = {"n": nn, "forward_us_per_iter": fwd * 1e6 / (K + 1), "backward_us_per_iter": bwd * 1e6 / (K + 1),
               "plain_us_per_iter": plain * 1e6 / K,
               "forward_amp_updates_per_s": N * K / fwd, "backward_amp_updates_per_s": N * K / bwd,
               "forward_over_plain": (fwd / (K + 1)) / (plain / K),
               "backward_over_plain": (bwd / (K + 1)) / (plain / K)}
        if hbm and nn >= 28:
            row["forward_hbm_frac"] = 16.0 * N * (K + 1) / fwd / 1e9 / hbm
            row["backward_hbm_frac"] = 32.0 * N * (K + 1) / bwd / 1e9 / hbm
            row["peak"] = f"{hbm} GB/s ({peak_src})"
        sizes.append(row)
        del s2, lam2
        torch.cuda.empty_cache()
    return {"study": "phase", "workload": f"n={n}, M={m} (seed {seed}), K={K}, phases U(0, 2pi) (seed {seed + 1}), "
            "uniform start, complex64",
            "loss_gpu": L_gpu, "loss_fp64": L_ref, "loss_err": abs(L_gpu - L_ref),
            "grad_scale": scale, "grad_max_err_vs_fp64_fd": err_fp64, "grad_max_err_vs_gpu_fd_h1e-4": fd_err,
            "adam_steps": 200, "adam_lr": 0.05, "adam_seconds": adam_s, "loss_initial": L_ref,
            "loss_final": final, "loss_final_fp64": final_ref, "p_final": math.exp(-final_ref),
            "p_bound_zalka": math.sin((2 * K + 1) * theta) ** 2, "timing": sizes}


def _timed_events(fn, reps, stream):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3 / reps


def run_phase_kernels(args):
    """The phase iterator's passes where they are HBM-bound: n=26 complex64
    (512 MiB state, 512 MiB adjoint), M=3, K=4, uniform start; forward and
    backward sweeps timed with CUDA events; bytes per pass: forward 16 B per
    amplitude (read + write), backward 32 B (state and adjoint)."""
    import numpy as np
    import torch
    from paper_2005_04635_gb300 import binding, inputs
    torch.cuda.set_device(0)
    binding.lib()
    n, m, K, seed = 26, 3, 4, 750
    N = 1 << n
    mk = binding.Marked(n, inputs.marked_indices(n, m, seed))
    phi, vphi = [torch.as_tensor(x, device="cuda") for x in inputs.uniform_phases(K, seed + 1)]
    stream = torch.cuda.current_stream()
    st = binding.State(n, "c64", stream=stream)
    lam = torch.empty(N, dtype=torch.complex64, device="cuda")
    gp = torch.empty(K, dtype=torch.float64, device="cuda")
    gv = torch.empty(K, dtype=torch.float64, device="cuda")
    st.init_uniform()
    for _ in range(args.warmup):
        st.phase_forward(mk, phi, vphi, None)
        st.phase_backward(mk, phi, vphi, lam, gp, gv)
    fwd = _timed_events(lambda: st.phase_forward(mk, phi, vphi, None), args.steps, stream)
    both = _timed_events(lambda: (st.phase_forward(mk, phi, vphi, None),
                                  st.phase_backward(mk, phi, vphi, lam, gp, gv)), args.steps, stream)
    st.sync()
    bwd = both - fwd
    peaks, src = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    # forward: one read-only reduction (8 B / amp) + K update passes (16 B);
    # backward: one start pass (read psi, write lambda: 16 B) + K passes (32 B)
    fwd_bytes = N * (8 + 16 * K)
    bwd_bytes = N * (16 + 32 * K)
    return {"study": "phase-kernels", "workload": f"n={n} complex64, M={m} (seed {seed}), K={K}, uniform start",
            "forward_ms": fwd * 1e3, "backward_ms": bwd * 1e3,
            "forward_gbs": fwd_bytes / fwd / 1e9, "backward_gbs": bwd_bytes / bwd / 1e9,
            "forward_frac": fwd_bytes / fwd / 1e9 / hbm, "backward_frac": bwd_bytes / bwd / 1e9 / hbm,
            "peak": f"{hbm} GB/s ({src})"}


def run_gate_kernels(args):
    """The conventional circuit where it is HBM-bound: n = --gate-n (default
    26, 512 MiB) complex64, M=1, uniform start; per-iteration time of
    grover_iterate_gate on each engine (oracle + 2 x the Walsh-Hadamard passes
    of one H^{(x)n}) with CUDA events, and the passes' GB/s."""
    import torch
    from paper_2005_04635_gb300 import binding, inputs
    torch.cuda.set_device(0)
    binding.lib()
    n, m, seed = args.gate_n, 1, 2601
    N = 1 << n
    mk = binding.Marked(n, inputs.marked_indices(n, m, seed))
    stream = torch.cuda.current_stream()
    out = {"study": "gate-kernels", "workload": f"n={n} complex64, M={m} (seed {seed}), uniform start"}
    for name, eng in (("tensor_cores", 1), ("cuda_cores", 0), ("default", -1)):
        st = binding.State(n, "c64", stream=stream)
        st.set_gate_engine(eng)
        st.init_uniform()
        for _ in range(args.warmup):
            st.iterate_gate(mk, 1)
        t = _timed_events(lambda: st.iterate_gate(mk, 1), args.steps, stream)
        st.sync()
        groups, on_tc = gate_engine_groups(n, eng)
        passes = 2 * len(groups)
        out[name] = {"iteration_ms": t * 1e3, "groups": groups, "tensor_cores": on_tc, "passes": passes,
                     "pass_gbs": passes * 16 * N / t / 1e9}
        del st
    return out


def run_batch_classes(args):
    """The batched workload's instance classes (n = 15-16, 17-18, 19, 20 of the
    seeded 4096-instance batch), or with --batch-n one class of --batch-count
    seeded instances of that size: each timed with CUDA events under each
    packing -- one CTA per instance (tuned), groups of CTAs holding the state
    in shared memory, clusters of 16 CTAs -- with P_success against the closed
    form."""
    import math
    import torch
    from paper_2005_04635_gb300 import binding, inputs
    torch.cuda.set_device(0)
    binding.lib()
    if args.batch_n:
        g = inputs.rng(4200 + args.batch_n)
        n = args.batch_n
        ms = [int(x) for x in g.integers(1, 9, args.batch_count)]
        marks = [inputs.marked_indices(n, m, 4300 + i) for i, m in enumerate(ms)]
        ks = [int(math.floor(0.78539816339744830962 * math.sqrt((1 << n) / m))) for m in ms]
        classes = {f"n{n}": ([n] * len(ms), ks, marks)}
    else:
        ns, ks, marks = batched_instances()
        classes = {}
        for lo, hi in ((15, 16), (17, 18), (19, 19), (20, 20)):
            sel = [i for i, n in enumerate(ns) if lo <= n <= hi]
            classes[f"n{lo}-{hi}"] = ([ns[i] for i in sel], [ks[i] for i in sel], [marks[i] for i in sel])
    stream = torch.cuda.current_stream()
    out = {"study": "batch-classes"}
    for name, (cn, ck, cm) in classes.items():
        b = binding.Batch(cn, ck, cm, stream=stream)
        b.tune()
        rec = {"instances": len(cn), "amp_updates": float(sum((1 << n) * k for n, k in zip(cn, ck))),
               "tuned_packing": b.packing()}
        for label, pk, mq in (("one_cta", 0, 17), ("groups", 2, 15), ("clusters", 16, 17)):
            if pk == 16 and max(cn) < 17:
                continue
            b.set_packing(pk, mq)
            for _ in range(args.warmup):
                b.run()
            t = _timed_events(b.run, args.steps, stream)
            p = b.success()
            err = max(abs(pi - p_success_closed_form(n, len(mk), k)) for pi, n, mk, k in zip(p, cn, cm, ck))
            rec[label] = {"ms": t * 1e3, "value": rec["amp_updates"] / t, "max_p_success_err": err}
        b.close()
        out[name] = rec
    return out


# ---- reference arm: the oracle on the host cores -----------------------------------------------------
def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return None
    import oracle
    from paper_2005_04635_gb300 import inputs
    if args.workload == "batched-4096":
        return run_reference_batched(args, world)
    w = workload(args.workload)
    n_s, iters = 24, 2  # bounded sample of the workload: 2^24 amplitudes, 2 iterations per step
    marked = inputs.marked_indices(n_s, min(w["M"], 1 << n_s), w["seed"])
    psi = oracle.init_uniform(n_s)
    for _ in range(args.warmup):
        oracle.grover_operator(psi, n_s, marked, iters)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.grover_operator(psi, n_s, marked, iters)
    dt = time.perf_counter() - t0
    value = (1 << n_s) * iters * args.steps / dt
    sample = (f"each step: n={n_s} (2^{n_s} complex128 amplitudes), M={len(marked)}, {iters} iterations of the "
              f"FP64 operator oracle (plain C, one thread), standing in for the {w['name']} workload")
    cfg = config_of(w, world)
    cfg["workload"] = (f"bounded sample of the {w['name']} workload: n={n_s} complex128 (FP64 oracle), "
                       f"M={len(marked)}, uniform init, {iters} iterations per step")
    cfg["sample"] = {"n": n_s, "state_dtype": "c128", "M": len(marked), "iterations_per_step": iters,
                     "state_bytes": (1 << n_s) * 16}
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded marked indices, uniform initial state)", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu_model(), "host_cores": host_cores()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_reference_batched(args, world):
    """The oracle on a bounded sample of the batched workload: per step, the
    first instances of the seeded batch with n <= 14, run to their optimal k."""
    import oracle
    ns, ks, marks = batched_instances()
    sample = [(n, k, mk) for n, k, mk in zip(ns, ks, marks) if n <= 14][:24]

    def step():
        for n, k, mk in sample:
            oracle.grover_operator(oracle.init_uniform(n), n, mk, k)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    units = float(sum((1 << n) * k for n, k, _ in sample)) * args.steps
    value = units / dt
    desc = f"each step: {len(sample)} instances of the seeded batch with n <= 14, FP64 operator oracle, one thread"
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (4096 seeded instances, uniform initial states)",
            "config": {"workload": f"bounded sample of the batched workload (4096 independent searches, n ~ U[8,20], "
                                   f"M ~ U[1,8]): {len(sample)} instances with n <= 14 per step",
                       "name": "batched-4096", "sample": {"instances": len(sample), "n_max": 14}},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc,
                             "cpu_model": cpu_model(), "host_cores": host_cores()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["batched-4096"], default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-n28", dest="n28", action="store_false",
                    help="skip the n = 28 full-search records of the default line")
    ap.add_argument("--batch-n", type=int, default=0, help="batch-classes study: one class of this size")
    ap.add_argument("--batch-count", type=int, default=16, help="batch-classes study: instances of that class")
    ap.add_argument("--study", choices=["precision", "phase", "phase-kernels", "gate-kernels", "batch-classes"],
                    default=None,
                    help="run a study instead of the throughput benchmark")
    ap.add_argument("--gate-n", type=int, default=26, help="qubits of the gate-kernels study")
    ap.add_argument("--gate-iters", type=int, default=2,
                    help="iterations of the conventional circuit timed for comparison (0: skip)")
    ap.add_argument("--path", choices=["auto", "pass", "resident"], default="auto",
                    help="auto: persistent on-chip iterator for small states, else one pass per iteration")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.study == "precision":
        out = run_precision_study(args)
    elif args.study == "phase":
        out = run_phase_study(args)
    elif args.study == "phase-kernels":
        out = run_phase_kernels(args)
    elif args.study == "gate-kernels":
        out = run_gate_kernels(args)
    elif args.study == "batch-classes":
        out = run_batch_classes(args)
    elif args.workload == "batched-4096" and args.impl != "reference":
        out = run_batched(args)
    else:
        out = run_reference(args) if args.impl == "reference" else run_ours(args)
    if out is not None:
        print(json.dumps(out), flush=True)
    try:
        import torch.distributed as dist
        if dist.is_available() and dist.is_initialized():
            dist.destroy_process_group()
    except Exception:
        pass


if __name__ == "__main__":
    main()
