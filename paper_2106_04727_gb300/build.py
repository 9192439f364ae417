"""Build the GB300 HAC library (libhac.so) in-tree with nvcc for sm_103a.

Each .cu under csrc/ compiles to an object in parallel; the objects link into
one shared library exporting the C ABI of include/hac.h.  No torch extension
machinery is involved: the library is plain CUDA C++ behind ``extern "C"``.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libhac.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC, *extra]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(INCLUDE, "hac.h"),
                                                                   os.path.abspath(__file__)]
    return any(os.path.getmtime(p) > t for p in deps)


def variant_dir(defines) -> str:
    """Build folder of a compiled variant (the tuner's tile shapes)."""
    tag = "_".join(f"{k}-{v}" for k, v in sorted(defines.items()))
    return os.path.join(BUILD, "variants", tag)


def build(force: bool = False, verbose: bool = False, ptxas_v: bool = False,
          defines=None) -> str:
    """Compile and link libhac.so if any source is newer than it.  With
    `defines` (macro -> value: the tile shapes of the tuner), a variant is
    built in its own folder and its path returned; the default library is
    untouched."""
    out_dir = variant_dir(defines) if defines else BUILD
    lib = os.path.join(out_dir, "libhac.so")
    if not force and not defines and not _stale():
        return LIB
    if defines and not force and os.path.exists(lib) and \
            all(os.path.getmtime(p) <= os.path.getmtime(lib)
                for p in sources() + glob.glob(os.path.join(CSRC, "*.cuh"))):
        return lib
    os.makedirs(out_dir, exist_ok=True)
    nv = nvcc()
    extra = ["-Xptxas", "-v"] if ptxas_v else []
    extra += [f"-D{k}={v}" for k, v in sorted((defines or {}).items())]

    def compile_one(src):
        obj = os.path.join(out_dir, os.path.basename(src)[:-3] + ".o")
        cmd = [nv, *_flags(extra), "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose or ptxas_v:
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=max(1, min(16, os.cpu_count() or 1, len(sources())))) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = lib + f".{os.getpid()}.tmp"
    r = subprocess.run([nv, *ARCH, "-shared", "-o", tmp, *objs],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


PROBE_SRC = os.path.join(HERE, "probe", "fma_probe.cu")
PROBE_LIB = os.path.join(BUILD, "libhacprobe.so")


def build_probe(force: bool = False) -> str:
    """The FP32 multiply-add throughput probe the benchmark uses as its
    arithmetic peak (a separate library; not part of the clustering ABI)."""
    if not force and os.path.exists(PROBE_LIB) and \
            os.path.getmtime(PROBE_LIB) >= os.path.getmtime(PROBE_SRC):
        return PROBE_LIB
    os.makedirs(BUILD, exist_ok=True)
    tmp = PROBE_LIB + f".{os.getpid()}.tmp"
    r = subprocess.run([nvcc(), *_flags(), "-shared", "-o", tmp, PROBE_SRC],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {PROBE_SRC}:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, PROBE_LIB)
    return PROBE_LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_v="-v" in sys.argv))
    print(build_probe(force="--force" in sys.argv))
