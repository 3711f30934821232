"""Build the C-ABI library ``libcosmo_du.so`` in-tree for sm_103a (B300).

    python -m paper_2606_13825_b300.build [--debug]

nvcc cross-compiles without a GPU.  The library is one translation unit
(``csrc/runtime.cu`` includes the kernel headers) linked against the static
CUDA runtime, so it carries no dependency on a particular libcudart path.
"""
import argparse
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libcosmo_du.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    src = os.path.join(HERE, "csrc")
    return [os.path.join(src, f) for f in sorted(os.listdir(src))
            if f.endswith((".cu", ".cuh", ".h"))] + [os.path.join(ROOT, "include", "cosmo_du.h")]


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in sources())


def build(debug=False, verbose=False, force=False):
    if not force and not debug and up_to_date():
        return LIB
    cmd = [nvcc_path(), *ARCH, "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-shared",
           "-cudart", "static", "-o", LIB + ".tmp", os.path.join(HERE, "csrc", "runtime.cu"),
           "-I", os.path.join(ROOT, "include")]
    cmd += ["-O0", "-G"] if debug else ["-O3"]
    if os.environ.get("COSMO_SPLIT_COMPILE") == "1":
        # device optimisation in parallel over the host's cores: a quicker
        # build for development; measured about 9% slower PSD kernels, so the
        # default build is one partition
        cmd += ["-split-compile=0"]
    if verbose:
        cmd += ["-Xptxas", "-v"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        sys.stderr.write(res.stdout + res.stderr)
        raise RuntimeError("nvcc failed building libcosmo_du.so")
    if verbose:
        sys.stderr.write(res.stderr)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--debug", action="store_true")
    ap.add_argument("--verbose", action="store_true")
    ap.add_argument("--force", action="store_true")
    a = ap.parse_args()
    print(build(debug=a.debug, verbose=a.verbose, force=a.force))
