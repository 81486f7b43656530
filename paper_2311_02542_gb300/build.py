"""Builds the CUDA library in-tree for sm_103a (GB300) with nvcc.

    python -m paper_2311_02542_gb300.build

compiles every csrc/*.cu to an object in parallel and links
_build/libvrnerf.so against the shared CUDA runtime (the one PyTorch loads).
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libvrnerf.so")
BUILD_CHECKED = BUILD + "_checked"
LIB_CHECKED = os.path.join(BUILD_CHECKED, "libvrnerf_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def cuda_lib_dir() -> str:
    root = os.path.dirname(os.path.dirname(os.path.realpath(nvcc())))
    for d in ("lib64", "targets/x86_64-linux/lib", "targets/sbsa-linux/lib", "lib"):
        p = os.path.join(root, d)
        if os.path.exists(os.path.join(p, "libcudart.so")):
            return p
    return os.path.join(root, "lib64")


def flags(extra=()):
    return [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
            "-Xptxas", "-warn-spills", *extra]


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    deps = [src] + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(HERE, "..", "include", "*.h"))
    return any(os.path.getmtime(d) > os.path.getmtime(obj) for d in deps)


def _link(objs, lib, force):
    if force or not os.path.exists(lib) or any(os.path.getmtime(o) > os.path.getmtime(lib) for o in objs):
        tmp = lib + f".{os.getpid()}.tmp"
        libdir = cuda_lib_dir()
        cmd = [nvcc(), *ARCH, "-shared", "-cudart", "shared", *objs, "-o", tmp, f"-L{libdir}",
               "-Xlinker", f"-rpath,{libdir}"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)


def build(verbose: bool = False, force: bool = False, checked: bool = True) -> str:
    """Compiles the release library and (checked=True) the checked one, whose
    device code verifies its indices (VRNERF_CHECKED=1), in one parallel pass."""
    os.makedirs(BUILD, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    cc = nvcc()
    variants = [(BUILD, LIB, [])]
    if checked:
        os.makedirs(BUILD_CHECKED, exist_ok=True)
        variants.append((BUILD_CHECKED, LIB_CHECKED, ["-DVRNERF_CHECKED=1"]))
    jobs = [(src, os.path.join(d, os.path.basename(src)[:-3] + ".o"), extra) for d, _, extra in variants
            for src in srcs]

    def compile_one(job):
        src, obj, extra = job
        if force or _stale(obj, src):
            cmd = [cc, *flags(extra), "-c", src, "-o", obj]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
            if verbose and (r.stdout or r.stderr):
                print(r.stdout + r.stderr, file=sys.stderr)
        return obj

    # the heaviest translation units first, so the pool stays busy
    jobs.sort(key=lambda j: -os.path.getsize(j[0]))
    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, jobs))
    for d, lib, _ in variants:
        _link([o for o in objs if os.path.dirname(o) == d], lib, force)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv))
