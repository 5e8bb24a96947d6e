"""Builds the in-tree CUDA library paper_2111_10270_gb300/_build/libfastdog.so
for sm_103a with nvcc (one translation unit per source, compiled in
parallel, then linked).  No cmake, no torch extension machinery."""
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
LIB = os.path.join(BUILD, "libfastdog.so")
INCLUDE = os.path.join(ROOT, "include")

SOURCES = ["bdd_build.cpp", "jit.cpp", "kernels.cu", "sweep_w2.cu", "sweep_w4.cu", "sweep_w8.cu", "sweep_w16.cu",
           "engine.cu", "batch.cu", "server.cu", "api.cu", "state.cu", "noalloc.cu", "eval.cu", "shard.cu", "persist.cu", "serial.cu", "plan_device.cu", "split.cpp", "host_pool.cpp"]
GEN = os.path.join(BUILD, "gen")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path() -> str:
    for cand in (os.environ.get("CUDA_HOME"), os.environ.get("CUDA_PATH"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "bin", "nvcc")):
            return os.path.join(cand, "bin", "nvcc")
    found = shutil.which("nvcc")
    if not found:
        raise RuntimeError("nvcc not found: set CUDA_HOME")
    return found


def _flags():
    return ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC,-O3", "-I", INCLUDE, "-I", CSRC, "-I", GEN]


def write_jit_sources():
    """Embeds the device-ABI block of fdog_internal.h and the kernel skeleton
    as string literals for the shape-specialised (NVRTC) kernels."""
    hdr = open(os.path.join(CSRC, "fdog_internal.h")).read()
    abi = hdr[hdr.index("// <jit-abi>"):hdr.index("// </jit-abi>")]
    skel = open(os.path.join(CSRC, "jit_skeleton.cuh")).read()
    os.makedirs(GEN, exist_ok=True)
    text = ("// generated by build.py from fdog_internal.h and jit_skeleton.cuh\n"
            f'static const char* kJitAbi = R"FDOGJIT({abi})FDOGJIT";\n'
            f'static const char* kJitSkeleton = R"FDOGJIT({skel})FDOGJIT";\n')
    path = os.path.join(GEN, "jit_sources.inc")
    if not os.path.exists(path) or open(path).read() != text:
        with open(path, "w") as f:
            f.write(text)


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "fastdog.h"))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force: bool = False, verbose: bool = False, ptxas_verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    nvcc = nvcc_path()
    write_jit_sources()
    obj_dir = os.path.join(BUILD, "obj")
    os.makedirs(obj_dir, exist_ok=True)
    flags = _flags()
    if ptxas_verbose:
        flags += ["-Xptxas", "-v"]

    def compile_one(src):
        obj = os.path.join(obj_dir, src + ".o")
        cmd = [nvcc, *flags, "-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cpp"):
            cmd = [nvcc, *flags, "-x", "c++", "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose:
        for _, log in results:
            if log.strip():
                sys.stderr.write(log)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *[o for o, _ in results], "-lcudart_static", "-lnvrtc", "-lrt", "-lpthread",
           "-ldl", "-Xlinker", "-rpath=" + os.path.join(os.path.dirname(os.path.dirname(nvcc)), "lib64")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_verbose="-v" in sys.argv)
    print(LIB)
