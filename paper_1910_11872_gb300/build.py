"""Build the CUDA library in-tree: nvcc, sm_103a only, one object per translation unit compiled
in parallel, linked into ``paper_1910_11872_gb300/_lib/librmusic.so``. ``build(checked=True)``
builds the checked variant (-DRMUSIC_CHECKS: the solvers test their work items' indices and
count failures instead of faulting) into ``_lib_checked/`` from objects in ``_build_checked/``."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "librmusic.so")
CHECKED_BUILD = os.path.join(HERE, "_build_checked")
CHECKED_LIB = os.path.join(HERE, "_lib_checked", "librmusic.so")
SOURCES = ["analytic.cu", "plain.cu", "batched.cu", "batched_l2_l4.cu", "batched_l6.cu", "batched_l8.cu",
           "batched_l10.cu", "batched_l12.cu", "batched_fwd.cu", "batched_fwd_l2_l5.cu", "batched_fwd_l6_l7.cu",
           "batched_fwd_l8.cu", "batched_fwd_l9_l10.cu", "batched_fwd_l11_l12.cu", "batched_p.cu",
           "batched_p_l3_l6.cu", "batched_p_l7_l9.cu", "batched_p_l10_l12.cu", "square.cu", "square_l1_l2.cu", "square_l3_l4.cu", "square_l5.cu",
           "square_l6.cu", "square_l7.cu", "square_l8.cu", "unwrap.cu", "crossband.cu", "capi.cu", "noalloc.cu", "serve.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ARCH + ["-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _inputs() -> list[str]:
    files = [os.path.join(CSRC, s) for s in SOURCES]
    files += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    files.append(os.path.join(os.path.dirname(HERE), "include", "rmusic.h"))
    return files


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    lib_path = CHECKED_LIB if checked else LIB
    build_dir = CHECKED_BUILD if checked else BUILD
    flags = FLAGS + (["-DRMUSIC_CHECKS"] if checked else [])
    if not force and up_to_date(lib_path):
        return lib_path
    os.makedirs(build_dir, exist_ok=True)
    os.makedirs(os.path.dirname(lib_path), exist_ok=True)
    cc = nvcc()

    def compile_one(src: str) -> tuple[str, str]:
        obj = os.path.join(build_dir, src.replace(".cu", ".o"))
        cmd = [cc] + flags + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    with open(os.path.join(build_dir, "ptxas.log"), "w") as f:
        for (obj, log), src in zip(results, SOURCES):
            f.write(f"==== {src}\n{log}\n")
    tmp = lib_path + f".{os.getpid()}.tmp"
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in results]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib_path)
    if verbose:
        print(open(os.path.join(build_dir, "ptxas.log")).read())
    return lib_path


if __name__ == "__main__":
    print(build(force=True, verbose=True))
