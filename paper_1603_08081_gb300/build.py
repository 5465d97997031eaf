"""In-tree build of ``libfbf.so`` (the C-ABI library) for sm_103a.

``python -m paper_1603_08081_gb300.build`` compiles every ``csrc/*.cu`` and
``csrc/*.cpp`` with nvcc in parallel and links one shared library under
``paper_1603_08081_gb300/_build/<machine>/``.  Objects are rebuilt when a source
or a header is newer.  No cmake, one ``-gencode``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import platform
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
ARCH_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a"]


def build_dir() -> str:
    return os.path.join(HERE, "_build", platform.machine())


def lib_path() -> str:
    return os.path.join(build_dir(), "libfbf.so")


def _nvcc() -> str:
    p = shutil.which("nvcc")
    if p:
        return p
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfbf.so")


def _cuda_lib_dir(nvcc: str) -> str:
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "lib64")


def _newest(paths) -> float:
    return max((os.path.getmtime(p) for p in paths), default=0.0)


def build(verbose: bool = False, force: bool = False) -> str:
    nvcc = _nvcc()
    out = build_dir()
    os.makedirs(out, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))
    headers = (glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
               + glob.glob(os.path.join(INCLUDE, "*.h")))
    hdr_t = _newest(headers)
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]
    jobs = []
    objs = []
    for s in srcs:
        o = os.path.join(out, os.path.basename(s) + ".o")
        objs.append(o)
        if force or not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(s), hdr_t):
            cmd = [nvcc] + ARCH_FLAGS + common
            if s.endswith(".cu"):
                cmd += ["-lineinfo", "-Xptxas", "-v"] if verbose else ["-lineinfo"]
            cmd += ["-c", s, "-o", o]
            jobs.append(cmd)

    def run(cmd):
        r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
        return cmd, r.returncode, r.stdout

    workers = max(1, min(len(jobs), os.cpu_count() or 4))
    failed = []
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        for cmd, rc, log in ex.map(run, jobs):
            if verbose or rc != 0:
                sys.stdout.write(" ".join(cmd[-3:]) + "\n" + log)
            if rc != 0:
                failed.append(cmd[-3])
    if failed:
        raise RuntimeError("nvcc failed for: " + ", ".join(failed))
    so = lib_path()
    if force or jobs or not os.path.exists(so):
        tmp = so + ".%d.tmp" % os.getpid()
        libdir = _cuda_lib_dir(nvcc)
        cmd = [nvcc] + ARCH_FLAGS + ["-shared", "-cudart", "shared", "-o", tmp] + objs + [
            "-Xlinker", "-rpath=" + libdir, "-L" + libdir, "-lcudart"]
        r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stdout)
        os.replace(tmp, so)
    return so


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
