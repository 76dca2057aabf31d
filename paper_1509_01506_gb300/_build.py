"""Builds libdnadfa.so in-tree with nvcc for sm_103a (GB300)."""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIBDIR = os.path.join(HERE, "_lib")
LIBPATH = os.path.join(LIBDIR, "libdnadfa.so")
SOURCES = [os.path.join(HERE, "csrc", f) for f in (
    "scan_inst_pair.cu", "scan_inst_one_smem.cu", "scan_inst_one_global.cu", "scan_inst_hot.cu", "scan_inst_one_rep.cu",
    "dna_scan.cu", "dna_batch.cu", "dna_map.cu", "dna_bench.cu", "dna_serve.cpp", "dna_compile.cpp", "dna_fasta.cpp")]
DEPS = SOURCES + [os.path.join(HERE, "csrc", f) for f in (
    "dna_internal.h", "dna_runtime.h", "dna_device.cuh", "scan_kernel.cuh")] + \
    [os.path.join(ROOT, "include", "dna_dfa.h")]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def up_to_date() -> bool:
    if not os.path.exists(LIBPATH):
        return False
    t = os.path.getmtime(LIBPATH)
    return all(os.path.getmtime(d) <= t for d in DEPS)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compiles each source to an object in parallel (one nvcc per file), then links."""
    if not force and up_to_date():
        return LIBPATH
    import concurrent.futures as cf
    os.makedirs(LIBDIR, exist_ok=True)
    tag = f"{os.getpid()}"
    objs = [os.path.join(LIBDIR, os.path.basename(src) + f".{tag}.o") for src in SOURCES]

    def compile_one(src, obj):
        cmd = [nvcc(), "-O3", "-std=c++17", "-Xcompiler", "-fPIC", ARCH, "-lineinfo", "-c", src, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        subprocess.check_call(cmd)

    try:
        with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
            for f in [ex.submit(compile_one, s, o) for s, o in zip(SOURCES, objs)]:
                f.result()
        tmp = LIBPATH + f".{tag}.tmp"
        subprocess.check_call([nvcc(), "-shared", ARCH, "-o", tmp] + objs)
        os.replace(tmp, LIBPATH)
    finally:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    return LIBPATH


if __name__ == "__main__":
    print(build(force=True, verbose=True))
