"""Build the CUDA library liblbm.so in-tree (paper_2208_04088_gb300/_build/).

sm_103a only: every .cu file is compiled with
``-gencode arch=compute_103a,code=sm_103a``; host C++ is compiled with
``-ffp-contract=off`` so the double-precision geometry tables are the same on
x86 and Arm hosts.  Translation units compile in parallel.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INC = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUT_DIR, "liblbm.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _cuda_home() -> str:
    home = os.environ.get("CUDA_HOME") or os.environ.get("CUDA_PATH")
    if home and os.path.exists(os.path.join(home, "bin", "nvcc")):
        return home
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    return "/usr/local/cuda"


def sources():
    cu = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))
    cpp = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cpp"))
    hdr = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".h"))
    hdr += [os.path.join(INC, f) for f in os.listdir(INC) if f.endswith(".h")]
    return cu, cpp, hdr


def _stale(out: str, deps) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def nvcc_flags(extra=()):
    return [ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
            "-I", INC, "-I", CSRC, *extra]


def build(force: bool = False, verbose: bool = False, extra_nvcc=()) -> str:
    cu, cpp, hdr = sources()
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and not _stale(LIB, cu + cpp + hdr + [os.path.abspath(__file__)]):
        return LIB
    home = _cuda_home()
    nvcc = os.path.join(home, "bin", "nvcc")
    jobs = []
    objs = []
    for src in cu:
        obj = os.path.join(OUT_DIR, os.path.basename(src) + ".o")
        objs.append(obj)
        jobs.append([nvcc, *nvcc_flags(extra_nvcc), "-c", src, "-o", obj])
    for src in cpp:
        obj = os.path.join(OUT_DIR, os.path.basename(src) + ".o")
        objs.append(obj)
        jobs.append(["g++", "-O3", "-std=c++17", "-fPIC", "-pthread", "-ffp-contract=off", "-Wall",
                     "-I", INC, "-I", CSRC, "-I", os.path.join(home, "include"), "-c", src,
                     "-o", obj])

    def run(cmd):
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"build failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        for log in ex.map(run, jobs):
            if verbose and log:
                print(log, file=sys.stderr)
    tmp = LIB + f".tmp{os.getpid()}"
    run([nvcc, ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-fPIC", "-lpthread"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
