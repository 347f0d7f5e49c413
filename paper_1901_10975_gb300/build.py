"""Build the engine's shared library in-tree (nvcc, sm_103a only)."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libcn.so")
SOURCES = [os.path.join(HERE, "csrc", f) for f in ("cn_engine.cu", "cn_solve.cu")]
DEPS = SOURCES + [os.path.join(HERE, "csrc", f) for f in ("cn_device.cuh", "cn_kernels.cuh")] + \
    [os.path.join(ROOT, "include", "cn.h")]


def nvcc_cmd(out, extra=()):
    return ["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo", "-O3", "-std=c++17",
            "-Xcompiler", "-fPIC", "-Xcompiler", "-pthread", "-shared", "--threads", "4", "-I", os.path.join(ROOT, "include"), *extra,
            "-o", out, *SOURCES]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in DEPS if os.path.exists(d))


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = nvcc_cmd(tmp, ("-Xptxas", "-v") if verbose else ())
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
