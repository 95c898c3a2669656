"""Builds librendermap.so in-tree (paper_1702_06813_gb300/_build/) with nvcc for sm_103a."""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "librendermap.so")
SOURCES = ["rm_api.cu", "rm_kernels.cu", "rm_noalloc.cu", "rm_normals.cu", "rm_mesh.cu", "rm_util.cu", "rm_vgrad.cu"]
HEADERS = ["rm_internal.cuh", "rm_kernels.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off",
         "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build librendermap")


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None,
          out_dir: str | None = None) -> str:
    """Compile every translation unit in parallel and link the shared library (into
    out_dir/librendermap.so when given, e.g. for a build with other -D knobs)."""
    build_dir = out_dir or BUILD
    lib = os.path.join(build_dir, "librendermap.so")
    os.makedirs(build_dir, exist_ok=True)
    nvcc = _nvcc()
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "rendermap.h")]
    objs = []
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(build_dir, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + hdrs):
            # each object goes to a private file first: processes that build at the same time
            # (one per GPU) never link a half-written object
            tmp_o = o + f".{os.getpid()}.tmp"
            cmd = [nvcc, *ARCH, *FLAGS, *(extra or []), "-c", s, "-o", tmp_o]
            jobs.append((cmd, tmp_o, o))
    if jobs:
        with concurrent.futures.ThreadPoolExecutor(len(jobs)) as ex:
            runs = ex.map(lambda j: subprocess.run(j[0], capture_output=True, text=True), jobs)
            for (cmd, tmp_o, o), res in zip(jobs, runs):
                if verbose or res.returncode != 0:
                    print(" ".join(cmd))
                    print(res.stdout + res.stderr)
                if res.returncode != 0:
                    raise RuntimeError(f"nvcc failed for {cmd[-3]}")
                os.replace(tmp_o, o)
    if force or jobs or _stale(lib, objs):
        tmp = lib + f".{os.getpid()}.tmp"
        res = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"],
                             capture_output=True, text=True)
        if res.returncode != 0:
            print(res.stdout + res.stderr)
            raise RuntimeError("link of librendermap.so failed")
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True))
