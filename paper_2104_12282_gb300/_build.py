"""Build libtomo.so (sm_103a) in-tree with nvcc: one object per .cu file, compiled in
parallel, linked into ``paper_2104_12282_gb300/_lib/libtomo.so``; with checked=True also
the bounds-checked variant ``libtomo_checked.so`` (-DTOMO_CHECKED)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
OBJ_DIR = os.path.join(OUT_DIR, "obj")
LIB = os.path.join(OUT_DIR, "libtomo.so")
LIB_CHECKED = os.path.join(OUT_DIR, "libtomo_checked.so")
SOURCES = ["api.cu", "element.cu", "matvec.cu", "matvec2.cu", "vec.cu", "filt.cu",
           "twoscale.cu", "server.cu", "noalloc.cu", "vtail.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", os.path.join(HERE, "..", "include")]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtomo")
    return exe


def _compile(src: str, extra, obj_dir: str) -> str:
    obj = os.path.join(obj_dir, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return obj


def _variants(checked: bool):
    """(library path, object directory, extra flags) of the regular build and, with
    checked, of the bounds-checked build (-DTOMO_CHECKED, libtomo_checked.so)."""
    out = [(LIB, OBJ_DIR, [])]
    if checked:
        out.append((LIB_CHECKED, os.path.join(OUT_DIR, "obj_checked"), ["-DTOMO_CHECKED"]))
    return out


def build(verbose: bool = False, extra=(), checked: bool = False) -> str:
    """Compile every source (all variants' translation units in one parallel pool), then
    link each variant; returns the regular library's path."""
    variants = _variants(checked)
    jobs = []
    for _, obj_dir, flags in variants:
        os.makedirs(obj_dir, exist_ok=True)
        jobs += [(s, list(extra) + flags, obj_dir) for s in SOURCES]
    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        objs = list(ex.map(lambda j: _compile(*j), jobs))
    for v, (lib, _, _) in enumerate(variants):
        part = objs[v * len(SOURCES):(v + 1) * len(SOURCES)]
        cmd = [nvcc(), *ARCH, "-shared", "-o", lib, *part, "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose:
            print(lib)
    return LIB


if __name__ == "__main__":
    args = [a for a in sys.argv[1:] if a != "--checked"]
    build(verbose=True, extra=args, checked="--checked" in sys.argv[1:])
