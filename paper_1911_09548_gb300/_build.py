"""Build the C-ABI shared library libstmg.so in-tree (CUDA for sm_103a + C++ host code).

    python -m paper_1911_09548_gb300._build

Compiles the translation units in parallel and links them with nvcc; the result is
paper_1911_09548_gb300/_lib/libstmg.so.  Rebuilds only when a source is newer.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_lib")
LIB_PATH = os.path.join(OUT_DIR, "libstmg.so")

CU_SOURCES = ["sn_kernels.cu", "sn_mixed.cu", "sn_dfc.cu", "sn_tc.cu", "st_kernels.cu", "tc_kernels.cu", "noalloc.cu"]
CPP_SOURCES = ["runtime.cpp", "mesh.cpp", "factor.cpp", "serve.cpp"]
GENCODE = "-gencode=arch=compute_103a,code=sm_103a"


def _cuda_home() -> str:
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("nvcc not found (set CUDA_HOME)")


def _sources():
    return [os.path.join(CSRC, s) for s in CU_SOURCES + CPP_SOURCES]


def _headers():
    return [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))] + [
        os.path.join(INCLUDE, h) for h in os.listdir(INCLUDE) if h.endswith(".h")]


def needs_build() -> bool:
    if not os.path.exists(LIB_PATH):
        return True
    t = os.path.getmtime(LIB_PATH)
    return any(os.path.getmtime(p) > t for p in _sources() + _headers() + [__file__])


def build(verbose: bool = False, force: bool = False) -> str:
    if not force and not needs_build():
        return LIB_PATH
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    obj_dir = os.path.join(OUT_DIR, "obj")
    os.makedirs(obj_dir, exist_ok=True)
    cmds = []
    objs = []
    for s in CU_SOURCES:
        o = os.path.join(obj_dir, s + ".o")
        objs.append(o)
        cmds.append([nvcc, GENCODE, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-I", CSRC, "-I", INCLUDE, "-c", os.path.join(CSRC, s), "-o", o])
    for s in CPP_SOURCES:
        o = os.path.join(obj_dir, s + ".o")
        objs.append(o)
        cmds.append(["g++", "-O3", "-std=c++17", "-fPIC", "-pthread", "-I", CSRC, "-I", INCLUDE,
                     "-I", os.path.join(cuda, "include"), "-c", os.path.join(CSRC, s), "-o", o])

    def run(cmd):
        p = subprocess.run(cmd, capture_output=True, text=True)
        if verbose or p.returncode:
            sys.stderr.write(" ".join(cmd) + "\n" + p.stdout + p.stderr)
        return p.returncode

    with ThreadPoolExecutor(max_workers=len(cmds)) as ex:
        rcs = list(ex.map(run, cmds))
    if any(rcs):
        raise RuntimeError("compilation of libstmg failed")
    tmp = LIB_PATH + ".tmp"
    link = [nvcc, GENCODE, "-shared", "-o", tmp] + objs + ["-Xcompiler", "-pthread"]
    if run(link):
        raise RuntimeError("linking libstmg failed")
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
