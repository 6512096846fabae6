"""Builds libadct.so in-tree with nvcc for sm_103a (translation units compiled in parallel)."""
from __future__ import annotations

import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libadct.so")
LIB_CHECKED = os.path.join(PKG, "libadct_checked.so")  # kernels with bounds checks (ADCT_CHECKED)
SOURCES = ["adct_api.cu", "adct_codec.cu", "adct_codec_zonal_lo.cu", "adct_codec_zonal_hi.cu",
           "adct_codec_interleaved.cu", "adct_codec_interleaved_edge.cu", "adct_codec_edge.cu", "adct_codec_masked.cu",
           "adct_codec_interleaved_masked.cu", "adct_float.cu",
           "adct_quality.cu", "adct_server.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libadct.so")


def _inputs():
    files = [os.path.join(CSRC, s) for s in SOURCES]
    files += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    files += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    files.append(os.path.abspath(__file__))
    return files


def up_to_date(checked: bool = False) -> bool:
    lib = LIB_CHECKED if checked else LIB
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compile every CUDA source for sm_103a and link libadct.so next to this
    file (checked: libadct_checked.so, whose kernels check their bounds)."""
    LIB_OUT = LIB_CHECKED if checked else LIB
    if not force and up_to_date(checked):
        return LIB_OUT
    nvcc = _nvcc()
    BUILD_DIR = os.path.join(BUILD, "checked") if checked else BUILD
    os.makedirs(BUILD_DIR, exist_ok=True)
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
    if checked:
        common += ["-DADCT_CHECKED"]
    procs = []
    objs = []
    for s in SOURCES:
        obj = os.path.join(BUILD_DIR, s.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [nvcc] + common + ["-Xptxas", "-v", "-c", os.path.join(CSRC, s), "-o", obj]
        log = open(os.path.join(BUILD_DIR, s + ".log"), "w")
        procs.append((subprocess.Popen(cmd, stdout=log, stderr=subprocess.STDOUT), log, s))
    failed = []
    for p, log, s in procs:
        rc = p.wait()
        log.close()
        if rc != 0:
            failed.append(s)
    if failed:
        msgs = "".join(open(os.path.join(BUILD_DIR, s + ".log")).read()[-4000:] for s in failed)
        raise RuntimeError(f"nvcc failed for {failed}:\n{msgs}")
    tmp = LIB_OUT + f".{os.getpid()}.tmp"
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "lib64")
    link = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-cudart", "shared", "-ldl", "-Xlinker", f"-rpath,{cuda_lib}"]
    subprocess.check_call(link)
    os.replace(tmp, LIB_OUT)
    if verbose:
        print("built", LIB_OUT)
    return LIB_OUT
