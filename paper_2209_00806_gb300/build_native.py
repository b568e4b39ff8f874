"""Build the CUDA library libtbpm.so in-tree for sm_103a (nvcc + g++).

Run as ``python paper_2209_00806_gb300/build_native.py`` (by path: importing the
package needs the library this script builds) or through
``__graft_entry__.build()``.  Output: ``paper_2209_00806_gb300/_build/libtbpm.so``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
SRC = PKG / "csrc"
OUT = PKG / "_build"
LIB = OUT / "libtbpm.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _nvcc() -> str:
    p = shutil.which("nvcc") or os.path.join(CUDA_HOME, "bin", "nvcc")
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA library cannot be built")
    return p


def sources():
    return sorted(SRC.glob("*.cu")) + sorted(SRC.glob("*.cpp"))


def _compile(src: Path, verbose_ptxas: bool) -> Path:
    obj = OUT / (src.name + ".o")
    if src.suffix == ".cu":
        cmd = [_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
               "--expt-relaxed-constexpr", "-I", str(PKG.parent / "include"), "-c", str(src),
               "-o", str(obj)]
        if verbose_ptxas:
            cmd.insert(1, "-Xptxas=-v")
    else:
        cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-fopenmp", "-I",
               os.path.join(CUDA_HOME, "include"), "-I", str(PKG.parent / "include"), "-c",
               str(src), "-o", str(obj)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    if verbose_ptxas:
        sys.stderr.write(r.stderr)
    return obj


def build(force: bool = False, verbose_ptxas: bool = False) -> Path:
    OUT.mkdir(exist_ok=True)
    srcs = sources()
    deps = srcs + [PKG.parent / "include" / "tbpm.h"] + sorted(SRC.glob("*.cuh"))
    if LIB.exists() and not force and not verbose_ptxas:
        t = LIB.stat().st_mtime
        if all(p.stat().st_mtime < t for p in deps):
            return LIB
    with ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose_ptxas), srcs))
    tmp = OUT / f"libtbpm.so.{os.getpid()}"
    cmd = [_nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", str(tmp),
           *map(str, objs), "-lgomp", "-Xlinker", "-rpath",
           "-Xlinker", os.path.join(CUDA_HOME, "lib64")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose_ptxas="-v" in sys.argv))
