"""Build the CUDA library libinterleaved_rans_b300.so in-tree (sm_103a).

    python -m paper_1402_3392_b300.build [--force] [--ptxas-verbose]

The shared object lands in paper_1402_3392_b300/_lib/ next to the binding
that loads it.  nvcc cross-compiles without a GPU.
"""
from __future__ import annotations

import argparse
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB_DIR = os.path.join(PKG, "_lib")
LIB_NAME = "libinterleaved_rans_b300.so"
LIB_PATH = os.path.join(LIB_DIR, LIB_NAME)
# The checked build (-DRANS_CHECKED): the kernels count failed invariants
# (rans_debug_checks in rans.h).  A test build, never the default.
LIB_PATH_CHECKED = os.path.join(LIB_DIR, "libinterleaved_rans_b300_checked.so")

SOURCES = ["rans_host.cpp", "rans_decode.cu", "rans_encode.cu", "rans_batch.cu", "rans_server.cu",
           "rans_check.cu", "rans_prefix.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _inputs():
    files = [os.path.join(CSRC, s) for s in SOURCES]
    files += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    files.append(os.path.join(INCLUDE, "rans.h"))
    files.append(os.path.abspath(__file__))
    return files


def is_stale(checked: bool = False) -> bool:
    path = LIB_PATH_CHECKED if checked else LIB_PATH
    if not os.path.exists(path):
        return True
    t = os.path.getmtime(path)
    return any(os.path.getmtime(f) > t for f in _inputs())


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def build(force: bool = False, ptxas_verbose: bool = False, quiet: bool = True,
          checked: bool = False) -> str:
    path = LIB_PATH_CHECKED if checked else LIB_PATH
    if not force and not ptxas_verbose and not is_stale(checked):
        return path
    os.makedirs(LIB_DIR, exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    cmd = [nvcc(), *ARCH, "-lineinfo", "-O3", "-std=c++17", "--expt-relaxed-constexpr",
           "-Xcompiler", "-fPIC,-O2,-Wall", "-shared", "-cudart", "shared",
           "-I", INCLUDE, "-I", CSRC, "-o", tmp]
    if ptxas_verbose:
        cmd += ["-Xptxas", "-v"]
    if checked:
        cmd += ["-DRANS_CHECKED"]
    cmd += [os.path.join(CSRC, s) for s in SOURCES]
    cmd += ["-Xlinker", "-rpath,/usr/local/cuda/lib64"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        sys.stderr.write(res.stdout + res.stderr)
        raise RuntimeError("nvcc failed building " + os.path.basename(path))
    if ptxas_verbose or not quiet:
        sys.stderr.write(res.stdout + res.stderr)
    os.replace(tmp, path)
    return path


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--ptxas-verbose", action="store_true")
    ap.add_argument("--checked", action="store_true", help="the checked test build")
    a = ap.parse_args(argv)
    print(build(force=a.force, ptxas_verbose=a.ptxas_verbose, quiet=False, checked=a.checked))


if __name__ == "__main__":
    main()
