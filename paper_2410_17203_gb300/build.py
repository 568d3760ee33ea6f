"""Build the CUDA library ``lib/libopfmp.so`` in-tree with nvcc for sm_103a.

The translation units are compiled in parallel, then linked against the
shared CUDA runtime so that a process that also loads PyTorch holds a single
runtime instance.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "lib", "libopfmp.so")
SOURCES = ["opf_kernels.cu", "opf_api.cu", "opf_wsnet.cu", "opf_diff.cu"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build the library")
    return exe


def cuda_lib_dir():
    root = os.path.dirname(os.path.dirname(os.path.realpath(nvcc())))
    return os.path.join(root, "lib64")


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(verbose=False, extra_flags=()):
    """Compile and link; returns the path of the shared library."""
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    common = [nvcc(), "-std=c++17", "-O3", ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
              "-I", INCLUDE, "-I", CSRC, *extra_flags]
    objs = [os.path.join(BUILD, s.replace(".cu", ".o")) for s in SOURCES]
    jobs = [common + ["-c", os.path.join(CSRC, s), "-o", o] for s, o in zip(SOURCES, objs)]
    with ThreadPoolExecutor(len(jobs)) as ex:
        outs = list(ex.map(_run, jobs))
    out = _run([nvcc(), ARCH, "-shared", "-cudart", "shared", "-o", LIB, *objs,
                "-Xlinker", "-rpath," + cuda_lib_dir()])
    if verbose:
        sys.stdout.write("".join(outs) + out)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
