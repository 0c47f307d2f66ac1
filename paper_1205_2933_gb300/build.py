"""Build the CUDA library libdwfmg.so in-tree for sm_103a (GB300).

Every .cu file under csrc/ is compiled in parallel with nvcc and linked into
paper_1205_2933_gb300/libdwfmg.so.  Objects live in paper_1205_2933_gb300/_build/.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import pathlib
import subprocess

PKG = pathlib.Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
INCLUDE = ROOT / "include"
BUILD = PKG / "_build"
LIB = PKG / "libdwfmg.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")


def _flags():
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", str(INCLUDE), "-I", str(CSRC)]


def _headers_mtime():
    hs = list(CSRC.glob("*.cuh")) + list(INCLUDE.glob("*.h"))
    return max(h.stat().st_mtime for h in hs)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> pathlib.Path:
    BUILD.mkdir(exist_ok=True)
    srcs = sorted(CSRC.glob("*.cu"))
    hm = _headers_mtime()
    jobs = []
    for s in srcs:
        o = BUILD / (s.stem + ".o")
        if force or ptxas_info or not o.exists() or o.stat().st_mtime < max(s.stat().st_mtime, hm):
            cmd = [NVCC] + _flags() + (["-Xptxas", "-v"] if ptxas_info else []) + ["-c", str(s), "-o", str(o)]
            jobs.append((s, cmd))

    def run(job):
        s, cmd = job
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed on {s.name}:\n{p.stderr}")
        return s.name, p.stderr

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            for name, err in ex.map(run, jobs):
                if verbose or ptxas_info:
                    print(f"[{name}]\n{err}")
    objs = [str(BUILD / (s.stem + ".o")) for s in srcs]
    if force or jobs or not LIB.exists():
        tmp = str(LIB) + ".tmp"
        subprocess.run([NVCC] + ARCH + ["-shared", "-o", tmp] + objs, check=True)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
