#!/usr/bin/env python
"""Throughput of the fixed-step cable-network engine on GB300.

Workload: the plain FP64 network -- 16,384 cells, each a random binary
dendritic tree of 200-600 compartments with an HH soma and passive dendrites,
50 ExpSyn per cell, 100 incoming NetCons per cell (delays 1-5 ms), 5 Hz
Poisson background per synapse, dt = 0.025 ms.  One benchmark step is one
minimum-delay interval (1 ms = 40 time steps) of the whole hot path: event
delivery, nrn_cur, matrix assembly, Hines solve, nrn_state, threshold
detection, and the spike exchange at the interval boundary.

Metric: compartment-updates/s = (sum of compartments) x 40 x steps / device
time, with every input resident in HBM; the model's working set (~0.6 GB)
is larger than L2, so no flush is needed between steps.

``--impl reference`` times the FP64 CPU oracle on the host cores on the same
workload (a bounded number of intervals), printing the same JSON line.
Under torchrun (N > 1) every rank runs an independent replica (the path is
single-GPU; replicas only).
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
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "compartment-updates/s on 1 GB300 at stated accuracy; fraction of HBM roofline"
UNIT = "compartment-updates/s"
B_ALG = 64.7            # algorithmic bytes per compartment-update (network workload)
FLOP_ALG = 15.0         # algorithmic FP64 flops per compartment-update (14 + 1 reciprocal)
FP64_PEAK_TFLOPS = 152 * 2.07e9 * 4 / 1e12   # 152 SMs x 2 FP64 FMA lanes/clk x 2 flop x 2.07 GHz
HBM_FALLBACK_GBS = 6800.0
KERNEL_SOURCES = ["paper_1901_10975_gb300/csrc/cn_kernels.cuh", "paper_1901_10975_gb300/csrc/cn_device.cuh"]


def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


def code_only(text):
    """Source text without comments and blank space, so that a digest changes
    with the code only (string literals in these sources hold no comment
    markers)."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_digest():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), encoding="utf-8") as fh:
            h.update(code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(args, mapping):
    """DRAM bytes per interval-kernel launch from the committed ncu summary of
    the full FP64 network workload, or None when this run is another workload
    or layout, or the kernel source changed since the capture."""
    if args.workload != "network" or args.cells not in (0, 16384) or args.precision != "fp64":
        return None
    p = os.path.join(ROOT, "profiles", "k_interval_network16k.md")
    try:
        txt = open(p).read()
    except OSError:
        return None
    m = re.search(r"kernel_digest:\s*([0-9a-f]+)", txt)
    if not m or m.group(1) != kernel_digest():
        return None
    t = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    lay = re.search(r"layout_mapping:\s*([0-9]+)", txt)
    if t and lay and int(lay.group(1)) == mapping:
        return float(t.group(1))
    for lm, tb in re.findall(r"layout_traffic:\s*([0-9]+)\s+([0-9.eE+]+)", txt):  # other layouts captured
        if int(lm) == mapping:
            return float(tb)
    return None


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload(args, intervals):
    if args.workload == "morph_types":
        from scenarios import morph_types
        return morph_types(n_cells=args.cells or 131072, cells_per_type=args.cells_per_type,
                           tstop=float(intervals) + 1.0)
    if args.workload == "batched":
        from scenarios import batched
        return batched(n_cells=args.cells or 50000, tstop=float(intervals) + 1.0, seed=1903)
    from scenarios import network
    return network(n_cells=args.cells or 16384, tstop=float(intervals) + 1.0, seed=1902)


def config_dict(args, sc, layout=None):
    cells = int(len(sc.cell_offset) - 1)
    if args.workload == "morph_types":
        name = (f"morphological types {cells} cells x 83 compartments, {args.cells_per_type} identical cells per "
                f"type, rings of 16, HH soma, pas dendrites, dt 0.025 ms")
    elif args.workload == "batched":
        name = (f"batched {cells} cells x lognormal(400, 0.8) compartments in [50, 5000], random subset of "
                f"6 channel types per cell on every node, network as the plain workload, dt 0.025 ms")
    else:
        name = (f"network {cells} cells x 200-600 compartments (HH soma, pas dendrites), "
                f"50 ExpSyn/cell, 100 NetCons/cell, 5 Hz background, dt 0.025 ms")
    d = {"workload": name, "cells": cells, "compartments": int(sc.n_nodes),
         "step": "one 1 ms min-delay interval (40 dt)", "l2": "working set > L2 (no flush needed)",
         "precision": args.precision}
    if layout is not None:
        mp, wpb, nw, tuned = layout
        span, height = mp & ((1 << 20) - 1), (mp >> 22) & 0x1ff
        tall = {1: ", tall warps", 2: ", warps twice the largest span", 3: ", warps 1.5 times the largest span"}.get(
            (mp >> 20) & 3, "")
        if height:
            tall = f", warps {height} rows tall"
        names = {1: "one cell per lane", 3: "reference: interleaved node ordering (one cell per lane)",
                 4: "reference: constant-depth node ordering (one node per lane and row)"}
        d["layout"] = {"mapping": names.get(mp, f"cells split to ~{span} rows per lane" + tall),
                       "mapping_value": int(mp), "warps_per_block": wpb, "warps": nw,
                       "chosen_by": "autotuner" if args.mapping == 2 else "fixed"}
    return d


def cpu_oracle_rate(sc, intervals, warm=0):
    """Oracle compartment-updates/s on all host cores over `intervals` ms."""
    from oracle import OracleModel
    sc.rec_node = sc.rec_node[:0]
    m = OracleModel(sc)
    threads = os.cpu_count() or 1
    if warm:
        m.run(warm * 40, threads)
    t0 = time.perf_counter()
    m.run(intervals * 40, threads)
    dt = time.perf_counter() - t0
    return sc.n_nodes * 40 * intervals / dt, threads, dt


def run_reference(args):
    world, rank, local = dist_setup()
    if world > 1 and rank != 0:
        return 0
    sc = workload(args, args.warmup + args.steps)
    t0 = time.perf_counter()
    rate, threads, dt = cpu_oracle_rate(sc, args.steps, warm=args.warmup)
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(args, sc),
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{args.steps} intervals ({args.steps * 40} steps) of the full "
                                       f"{args.workload} workload after {args.warmup} warm-up intervals"},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    world, rank, local = dist_setup()
    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_1901_10975_gb300 import build
    if rank == 0:
        build.build()
    barrier(world)
    from paper_1901_10975_gb300 import cn
    W, K = args.warmup, args.steps
    sc = workload(args, W + K)
    md = cn.from_scenario(sc, precision=args.precision, device=local, record=False, mapping=args.mapping,
                          warps_per_block=args.wpb)
    md.cn_profile(True)
    layout = md.cn_get_mapping()              # lays the model out (autotuned by default)
    md.cn_run(float(W))                       # warm-up intervals
    md.cn_sync()
    md.cn_profile_read()
    launches0 = md.launches
    barrier(world)
    torch.cuda.synchronize()
    clk = Clocks(local)
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    md.cn_run(float(W + K))
    e1.record()
    torch.cuda.synchronize()
    barrier(world)
    clocks = clk.stop()
    md.cn_sync()
    ms = e0.elapsed_time(e1)
    ms_max = max_over_ranks(ms, world)
    launches = md.launches - launches0
    k_ms, k_n, p_ms, p_n = md.cn_profile_read()
    updates = sc.n_nodes * 40 * K
    value = updates * world / (ms_max / 1e3)
    per_launch = k_ms / max(k_n, 1)
    upd_launch = sc.n_nodes * 40
    achieved_tflops = FLOP_ALG * upd_launch / (per_launch / 1e3) / 1e12
    hbm, hbm_kind = hbm_peak()
    traffic = profiled_traffic(args, layout[0] if layout is not None else -1)
    kernel_rate = upd_launch / (per_launch / 1e3)
    fp64_meas = md.fp64_peak()              # a DFMA stream on this GPU, TFLOP/s
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else f"f64 (gates {args.precision[5:]})",
        "data": "synthetic", "config": config_dict(args, sc, layout),
        "gpu_launches": int(launches),
        "roofline": {"bound": "alu", "pipe": "fp64", "achieved": achieved_tflops, "peak": FP64_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": achieved_tflops / FP64_PEAK_TFLOPS, "traffic": traffic,
                     "kernel": "k_interval", "kernel_ms_per_launch": per_launch,
                     "kernel_share": k_ms / ms, "peak_kind": "nominal (units x clock)",
                     "flops_per_update": FLOP_ALG, "peak_measured": fp64_meas,
                     "frac_of_measured": achieved_tflops / fp64_meas if fp64_meas else None},
        "hbm_roofline": {"bound": "hbm", "achieved": kernel_rate * B_ALG / 1e9, "peak": hbm, "unit": "GB/s",
                         "frac": kernel_rate * B_ALG / 1e9 / hbm, "bytes_per_update": B_ALG,
                         "peak_kind": hbm_kind, "whole_step_frac": value / world * B_ALG / 1e9 / hbm},
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_e2e:
        line["e2e"] = e2e_measure(args, cn, K, layout)
        if not args.no_e2e_full:  # the whole 1,000 ms run: setup amortised as in real use
            line["e2e_full_run"] = e2e_measure(args, cn, 1000, layout)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sc_cpu = workload(args, args.cpu_intervals)
        rate, threads, dt = cpu_oracle_rate(sc_cpu, args.cpu_intervals)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": f"first {args.cpu_intervals} intervals ({args.cpu_intervals * 40} steps) "
                                          f"of the full {args.workload} workload, {dt:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    md.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def e2e_measure(args, cn, K, layout):
    """Same metric through the public API from host buffers: model creation
    from pinned host arrays (geometry, tables, NetCons, events: the H2D
    copies), K intervals, then the spike raster and soma traces back to the
    host (D2H), all inside one wall-clock region."""
    import numpy as np
    import torch
    sc = workload(args, K)
    pin = {}
    for name in ("cell_offset", "parent", "dx", "diam", "Ra", "cm", "netcon_src", "netcon_syn", "netcon_w",
                 "netcon_delay", "ev_syn", "ev_t", "ev_w"):
        a = getattr(sc, name)
        t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        pin[name] = t
        setattr(sc, name, t.numpy())
    h2d = sum(t.numel() * t.element_size() for t in pin.values())
    h2d += sum(m.node.nbytes + m.param_matrix().nbytes for m in sc.mechs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    md = cn.from_scenario(sc, precision=args.precision, record=True, mapping=layout[0],
                          warps_per_block=layout[1])
    md.cn_run(float(K))
    g, k = md.cn_get_spikes()
    tr = md.cn_get_traces()
    dt = time.perf_counter() - t0
    d2h = g.nbytes + k.nbytes + tr.nbytes
    md.close()
    return {"value": sc.n_nodes * 40 * K / dt, "unit": UNIT, "h2d_bytes_per_step": h2d / K,
            "d2h_bytes_per_step": d2h / K, "seconds": dt,
            "intervals": K,
            "region": "cn_geometry + cn_model_create + cn_add_* + cn_run + cn_get_spikes + cn_get_traces "
                      "(with the layout the autotuner chose for the device-timed run)"}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100, help="timed 1 ms intervals")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cells", type=int, default=0, help="0: the workload's full size")
    ap.add_argument("--workload", choices=["network", "batched", "morph_types"], default="network")
    ap.add_argument("--cells-per-type", type=int, default=32, help="morph_types: identical cells per type")
    ap.add_argument("--precision", choices=["fp64", "gate_fp32", "gate_bf16"], default="fp64")
    ap.add_argument("--cpu-intervals", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--mapping", type=int, default=2,
                    help="2: autotuned, 0: split to the mean cell size, 1: one cell per lane, "
                         "3: reference interleaved layout, 4: reference constant-depth layout, "
                         ">=16: target rows per lane")
    ap.add_argument("--wpb", type=int, default=0,
                    help="warps per block of the interval kernel for a fixed --mapping (0: 1; the "
                         "autotuner picks its own)")
    ap.add_argument("--no-e2e-full", action="store_true",
                    help="skip the end-to-end timing of a whole 1,000 ms run through the public API")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
