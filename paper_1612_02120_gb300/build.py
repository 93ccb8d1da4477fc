"""Build step of libmembrane.so: nvcc for sm_103a only, one object per translation unit, compiled in
parallel, linked in-tree next to this file. Rebuilds only what changed."""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OBJ = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libmembrane.so")
SOURCES = ["api.cu", "simt_conv.cu", "tc_conv.cu", "student.cu", "noalloc.cu", "fastmemb.cu", "fastmemb_tc.cu", "maskextend.cu",
           "maskextend_tc.cu", "student_tc.cu"]
HEADERS = [os.path.join(CSRC, "internal.h"), os.path.join(CSRC, "tc_ptx.cuh"), os.path.join(CSRC, "simt_conv.cuh"),
           os.path.join(CSRC, "fm_conv.cuh"),
           os.path.join(ROOT, "include", "membrane.h")]

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
         "-Xcompiler", "-fPIC,-O2", "-Xptxas", "-v", "-I", os.path.join(ROOT, "include")]


def _mtime(p: str) -> float:
    return os.path.getmtime(p) if os.path.exists(p) else 0.0


def _compile(src: str) -> tuple[str, str]:
    s = os.path.join(CSRC, src)
    o = os.path.join(OBJ, src.replace(".cu", ".o"))
    newest_dep = max([_mtime(s)] + [_mtime(h) for h in HEADERS])
    if _mtime(o) >= newest_dep:
        return o, ""
    r = subprocess.run([NVCC, *FLAGS, "-c", s, "-o", o], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    return o, r.stderr


def build(verbose: bool = False) -> str:
    os.makedirs(OBJ, exist_ok=True)
    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(_compile, SOURCES))
    log = "".join(err for _, err in results)
    if log:
        with open(os.path.join(OBJ, "ptxas.log"), "w") as f:
            f.write(log)
        if verbose:
            sys.stderr.write(log)
    objs = [o for o, _ in results]
    if _mtime(LIB) < max(_mtime(o) for o in objs):
        tmp = LIB + f".{os.getpid()}.tmp"
        r = subprocess.run([NVCC, "-shared", "-o", tmp, *objs, "-lcuda"], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
