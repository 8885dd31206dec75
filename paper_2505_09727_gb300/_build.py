"""Compile the CUDA library libesp_gb300.so in-tree for sm_103a.

Translation units are compiled in parallel (nvcc for .cu, g++ for .cpp) and
linked with nvcc against cuFFT. Output: paper_2505_09727_gb300/_build/.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libesp_gb300.so")
# throughput microbenchmarks (roofline denominators), kept out of the solver library
PEAKS_LIB = os.path.join(OUT, "libesp_peaks.so")
PEAKS_SOURCE = "esp_peaks.cu"

ARCH = "-gencode=arch=compute_103a,code=sm_103a"
NVCC_FLAGS = [ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-Wno-deprecated-declarations", "--expt-relaxed-constexpr"]
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-Wall", "-pthread"]

CU_SOURCES = ["esp_kern_f32.cu", "esp_kern_f32_rest.cu", "esp_kern_near.cu", "esp_kern_f64.cu",
              "esp_kern_f64_rest.cu", "esp_plan.cu", "esp_engine.cu", "esp_static.cu", "esp_md.cu"]
CPP_SOURCES = ["esp_math.cpp", "esp_server.cpp", "esp_tune.cpp"]


def cuda_home() -> str:
    for cand in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "bin", "nvcc")):
            return cand
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    raise RuntimeError("nvcc not found")


def _sources_newer(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    deps = [src] + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    deps.append(os.path.join(HERE, "..", "include", "esp.h"))
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(verbose: bool = False, force: bool = False) -> str:
    home = cuda_home()
    nvcc = os.path.join(home, "bin", "nvcc")
    os.makedirs(OUT, exist_ok=True)
    jobs = []
    objs = []
    for src in CU_SOURCES + CPP_SOURCES:
        path = os.path.join(CSRC, src)
        obj = os.path.join(OUT, src.rsplit(".", 1)[0] + ".o")
        objs.append(obj)
        if not force and not _sources_newer(obj, path):
            continue
        if src.endswith(".cu"):
            cmd = [nvcc] + NVCC_FLAGS + ["-c", path, "-o", obj]
        else:
            cmd = ["g++"] + CXX_FLAGS + ["-I", os.path.join(home, "include"), "-c", path, "-o", obj]
        jobs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for cmd, proc in jobs:
        out, _ = proc.communicate()
        if verbose or proc.returncode:
            sys.stdout.write(out.decode(errors="replace"))
        if proc.returncode:
            failed.append(" ".join(cmd))
    if failed:
        raise RuntimeError("compilation failed:\n" + "\n".join(failed))
    peaks_src = os.path.join(CSRC, PEAKS_SOURCE)
    peaks_job = None
    if force or not os.path.exists(PEAKS_LIB) or os.path.getmtime(peaks_src) > os.path.getmtime(PEAKS_LIB):
        cmd = [nvcc] + NVCC_FLAGS + ["-shared", peaks_src, "-o", PEAKS_LIB]
        peaks_job = (cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT))
    if peaks_job:
        out, _ = peaks_job[1].communicate()
        if verbose or peaks_job[1].returncode:
            sys.stdout.write(out.decode(errors="replace"))
        if peaks_job[1].returncode:
            raise RuntimeError("compilation failed:\n" + " ".join(peaks_job[0]))
    if jobs or not os.path.exists(LIB):
        libdir = os.path.join(home, "lib64")
        cmd = [nvcc, ARCH, "-shared", "-o", LIB] + objs + [
            "-L" + libdir, "-lcufft", "-Xlinker", "-rpath=" + libdir]
        proc = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
        if proc.returncode:
            raise RuntimeError("link failed:\n" + proc.stdout.decode(errors="replace"))
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv))
