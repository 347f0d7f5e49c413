"""The multi-process side of bench.py on CPU (gloo, world size 2).

The engine does not shard (replicas only): under torchrun every rank runs
its own replica, the timing is the maximum over ranks, and the reference arm
runs on rank 0 alone.  These tests run that host logic without a GPU."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _max_worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, _ = bench.dist_setup()
    bench.barrier(w)
    out[r] = bench.max_over_ranks(10.0 + 5.0 * r, w)
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    import torch.multiprocessing as mp
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_max_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    assert dict(out) == {0: 15.0, 1: 15.0}


def test_reference_arm_under_torchrun_prints_once():
    """--impl reference under a 2-rank launch: rank 0 times the oracle on a
    bounded sample and prints one JSON line; rank 1 exits 0 without work."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "3", "--cells", "64"]
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


def test_kernel_digest_ignores_comments_only():
    """The digest that ties the ncu traffic in profiles/ to the kernel hashes
    code only: comments and blank space do not change it, code does."""
    sys.path.insert(0, ROOT)
    import bench
    a = "int f(int x) { // the input\n  return x + 1; /* one more */ }\n"
    b = "int f(int x) {\n\n  return x + 1;   }"
    c = "int f(int x) { return x + 2; }"
    assert bench.code_only(a) == bench.code_only(b)
    assert bench.code_only(a) != bench.code_only(c)
    assert "//" not in bench.code_only(a) and "/*" not in bench.code_only(a)


def test_profiled_traffic_only_for_its_layout():
    """The DRAM traffic of the committed ncu summary is reported only for the
    workload, precision and layout it was captured on, with the kernel source
    it was captured from."""
    import argparse
    import re
    sys.path.insert(0, ROOT)
    import bench
    txt = open(os.path.join(ROOT, "profiles", "k_interval_network16k.md")).read()
    mp = int(re.search(r"layout_mapping:\s*([0-9]+)", txt).group(1))
    digest = re.search(r"kernel_digest:\s*([0-9a-f]+)", txt).group(1)
    args = argparse.Namespace(workload="network", cells=0, precision="fp64")
    t = bench.profiled_traffic(args, mp)
    if digest == bench.kernel_digest():
        assert t is not None and t > 16.95e9  # at least the algorithmic bytes of a launch
    else:
        assert t is None
    assert bench.profiled_traffic(args, mp + 1) is None
    for lm, tb in re.findall(r"layout_traffic:\s*([0-9]+)\s+([0-9.eE+]+)", txt):
        if digest == bench.kernel_digest():
            assert bench.profiled_traffic(args, int(lm)) == float(tb)
    for other in (dict(workload="batched"), dict(cells=8192), dict(precision="gate_fp32")):
        assert bench.profiled_traffic(argparse.Namespace(**{**vars(args), **other}), mp) is None


def test_layout_description_names_the_warp_height():
    sys.path.insert(0, ROOT)
    import argparse
    import bench

    class Sc:
        n_nodes = 100
        cell_offset = [0, 50, 100]

    args = argparse.Namespace(workload="network", cells=0, precision="fp64", mapping=2, cells_per_type=32)
    d = bench.config_dict(args, Sc(), (32 | (1 << 20) | (112 << 22), 4, 2375, 6.5))
    assert d["layout"]["mapping"] == "cells split to ~32 rows per lane, warps 112 rows tall"
    assert d["layout"]["mapping_value"] == 32 | (1 << 20) | (112 << 22)
    d = bench.config_dict(args, Sc(), (43 | (1 << 20), 4, 2272, 7.6))
    assert d["layout"]["mapping"] == "cells split to ~43 rows per lane, tall warps"
