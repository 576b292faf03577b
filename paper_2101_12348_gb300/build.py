"""Builds libftp_gb300.so (the C-ABI library of include/ftp.h) for sm_103a.

Each CUDA translation unit is compiled by nvcc in parallel, then linked with
cuFFT into a shared library placed next to this file.  No CMake, no torch
extension machinery: the library is plain C ABI and is loaded with ctypes.

build(checks=True) makes the self-checking variant libftp_gb300_checks.so in
its own build folder: every guarded index and alignment check of the kernels
is compiled in (-DFTP_DEVICE_CHECKS); a failed check records its site in the
status block and skips the access instead of faulting.
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
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libftp_gb300.so")
BUILD_CHECKS = os.path.join(PKG, "_build_checks")
LIB_CHECKS = os.path.join(PKG, "libftp_gb300_checks.so")
SOURCES = ["ftp_api.cu", "ftp_nfft.cu", "ftp_roots_mixed.cu", "ftp_roots_fp64.cu",
           "ftp_roots_redo.cu", "ftp_noalloc.cu", "ftp_screen.cu", "ftp_mlp.cu",
           "ftp_mlp_api.cu", "ftp_shared.cu", "ftp_peaks.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def _flags(extra=(), checks_on=False):
    checks = ["-DFTP_DEVICE_CHECKS"] if checks_on else []
    return ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
            "-I", os.path.join(ROOT, "include"), *ARCH, *checks, *extra]


def _newer(dst: str, srcs) -> bool:
    if not os.path.exists(dst):
        return False
    t = os.path.getmtime(dst)
    return all(os.path.getmtime(s) <= t for s in srcs)


def build(verbose: bool = False, force: bool = False, ptxas_info: bool = False,
          checks: bool = False) -> str:
    """Compile (if stale) and return the path of the shared library (the
    self-checking variant with checks=True or FTP_DEVICE_CHECKS=1 set)."""
    checks = checks or os.environ.get("FTP_DEVICE_CHECKS") == "1"
    bdir, lib = (BUILD_CHECKS, LIB_CHECKS) if checks else (BUILD, LIB)
    os.makedirs(bdir, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(ROOT, "include", "ftp.h"))
    exe = nvcc()
    jobs = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(bdir, src.replace(".cu", ".o"))
        objs.append(o)
        if force or ptxas_info or not _newer(o, [s, *headers, __file__]):
            extra = ["-Xptxas", "-v"] if ptxas_info else []
            jobs.append([exe, *_flags(extra, checks), "-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            for cmd, r in ex.map(run, jobs):
                if verbose or ptxas_info:
                    sys.stderr.write(r.stdout + r.stderr)
                if r.returncode != 0:
                    raise RuntimeError(f"nvcc failed ({' '.join(cmd)}):\n{r.stdout}\n{r.stderr}")
    if force or jobs or not _newer(lib, objs):
        cmd = [exe, *ARCH, "-shared", "-o", lib, *objs, "-lcufft", "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    return lib


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv, ptxas_info="--ptxas" in sys.argv,
                checks="--checks" in sys.argv))
