"""Build ``libgbfft.so`` in-tree with nvcc for sm_103a (no cmake, no setuptools).

Regenerates the codelets if their generator changed, compiles every
translation unit in parallel into ``_build/`` and links one shared library
next to this file.  Nothing is rebuilt when the objects are up to date.
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
BUILD = os.path.join(ROOT, "_build", "gbfft")
LIB = os.path.join(HERE, "libgbfft.so")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", CSRC, "-I", INCLUDE]
SOURCES = ["stockham.cu", "group_kernel.cu", "stockham_pow2.cu", "tc.cu", "tables.cu", "bluestein.cu", "rader.cu", "real.cu", "plan.cpp", "builder.cpp", "api.cpp", "group.cpp", "server.cpp", "noalloc.cu", "cluster.cu", "l2fourstep.cu", "stockham_mr.cu", "stockham_mr512.cu", "stockham_mrc.cu", "stockham_mrc2.cu"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _headers():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".hpp", ".cuh"))] + \
        [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def generate_codelets():
    gen = os.path.join(CSRC, "gen_codelets.py")
    out = os.path.join(CSRC, "codelets.cuh")
    if _stale(out, [gen]):
        subprocess.check_call([sys.executable, gen, out])


def build(verbose: bool = False, jobs: int | None = None) -> str:
    generate_codelets()
    os.makedirs(BUILD, exist_ok=True)
    hdrs = _headers()
    cc = nvcc()
    jobs_list = []
    objs = []
    for src in SOURCES:
        path = os.path.join(CSRC, src)
        obj = os.path.join(BUILD, src + ".o")
        objs.append(obj)
        if _stale(obj, [path] + hdrs + [__file__]):
            cmd = [cc] + ARCH + COMMON + ["-c", path, "-o", obj]
            if src.endswith(".cu"):
                cmd += ["-Xptxas", "-warn-spills"]
            jobs_list.append(cmd)

    def run(cmd):
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError("compile failed:\n" + " ".join(cmd) + "\n" + p.stdout + p.stderr)
        return p.stdout + p.stderr

    if jobs_list:
        n = jobs or min(len(jobs_list), os.cpu_count() or 4)
        with concurrent.futures.ThreadPoolExecutor(max_workers=n) as ex:
            for out in ex.map(run, jobs_list):
                if verbose and out.strip():
                    print(out)
    if jobs_list or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        run([cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lpthread"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
