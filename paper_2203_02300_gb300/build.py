"""Build the sm_103a shared library libdco_stereo.so in-tree (csrc -> _lib).

One translation unit, one -gencode (compute_103a / sm_103a), plain nvcc:
no torch extension machinery, no cmake.  The result is git-ignored and
rebuilt on every machine (the GPU machine is aarch64, this container x86_64).
"""
import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIB_DIR, "libdco_stereo.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def nvcc_command(out: str, extra=()):
    return (["nvcc", *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
             f"-I{INCLUDE}", "-o", out] + list(extra) + _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(LIB_DIR, exist_ok=True)
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(f) <= t for f in _deps()):
            return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = nvcc_command(tmp, ["-Xptxas", "-v"] if verbose else [])
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
