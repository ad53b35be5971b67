"""Build the CUDA library ``libvstereo.so`` in-tree for sm_103a (B300).

    python -m paper_1902_09733_b300.build [--force]

Every ``csrc/*.cu`` is compiled by nvcc (one process per file, in parallel) for ``compute_103a/sm_103a`` and
linked into ``paper_1902_09733_b300/libvstereo.so`` next to this file, so the
built library travels with the source tree; the same sources with
``-DVS_CHECKED`` (bounds checks in the min-sum kernels, for tests) give
``libvstereo_checked.so``.  No GPU is needed to build.
"""
from __future__ import annotations

import concurrent.futures
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(HERE, "libvstereo.so")
CHECKED_LIB = os.path.join(HERE, "libvstereo_checked.so")
OBJ_DIR = os.path.join(HERE, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "--expt-relaxed-constexpr",
              "-Xptxas", "-v"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libvstereo.so")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(CHECKED_LIB):
        return True
    t = min(os.path.getmtime(LIB), os.path.getmtime(CHECKED_LIB))
    deps = sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    return any(os.path.getmtime(p) > t for p in deps)


SCENE_SRC = os.path.join(HERE, "scene", "vs_render.cu")
SCENE_LIB = os.path.join(HERE, "scene", "libvsrender.so")


def build_scene(force: bool = False) -> str:
    """The flight-scene renderer (test and benchmark input generation), a
    library of its own next to its source, compiled without fused
    multiply-adds so that it rounds as the host renderer does."""
    if not force and os.path.exists(SCENE_LIB) and os.path.getmtime(SCENE_LIB) >= os.path.getmtime(SCENE_SRC):
        return SCENE_LIB
    tmp = SCENE_LIB + f".{os.getpid()}.tmp"
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-Xcompiler", "-fPIC", "-shared",
           SCENE_SRC, "-o", tmp, "-lcudart_static", "-lrt", "-lpthread", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {SCENE_SRC}:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, SCENE_LIB)
    return SCENE_LIB


def build(force: bool = False, verbose: bool = False) -> str:
    build_scene(force)
    if not force and not _stale():
        return LIB
    os.makedirs(os.path.join(OBJ_DIR, "checked"), exist_ok=True)
    srcs = sources()
    # the product library and the checked build (-DVS_CHECKED, bounds checks in the min-sum kernels)
    jobs = [(src, os.path.join(OBJ_DIR, os.path.basename(src)[:-3] + ".o"), []) for src in srcs]
    jobs += [(src, os.path.join(OBJ_DIR, "checked", os.path.basename(src)[:-3] + ".o"), ["-DVS_CHECKED"])
             for src in srcs]

    def compile_one(job):
        src, obj, extra = job
        cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *extra, "-I", INCLUDE, "-c", src, "-o", obj]
        return subprocess.run(cmd, capture_output=True, text=True)

    # one nvcc per source file and build, in parallel
    with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        results = list(ex.map(compile_one, jobs))
    log = []
    for (src, _, extra), r in zip(jobs, results):
        if not extra:
            log.append(r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc {' '.join(extra)} failed on {src}:\n{r.stdout}\n{r.stderr}")
    for lib, objs in ((LIB, [j[1] for j in jobs if not j[2]]), (CHECKED_LIB, [j[1] for j in jobs if j[2]])):
        tmp = lib + f".{os.getpid()}.tmp"
        cmd = [nvcc(), *ARCH, "-shared", "-Xcompiler", "-fPIC", "-o", tmp, *objs, "-lcudart_static", "-lrt",
               "-lpthread", "-ldl"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    with open(os.path.join(OBJ_DIR, "ptxas.log"), "w") as f:
        f.write("\n".join(log))
    if verbose:
        print("\n".join(log))
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
