"""In-tree build of libheatcg.so for GB300 (sm_103a) with nvcc.

Objects compile in parallel; the shared library lands in
``paper_2608_11882_gb300/_build/libheatcg.so`` (git-ignored).  No torch
headers are involved: the library's ABI is plain C (include/heatcg.h).
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
BUILD = PKG / "_build"
LIB = BUILD / "libheatcg.so"
SOURCES = ["api.cu", "heat.cu", "heat_tb.cu", "heat_stream.cu", "heat_batch.cu", "heat_vk.cu", "cg.cu",
           "cg_spmv_tma.cu", "cg_mixed.cu", "cg_batch.cu"]
HEADERS = [ROOT / "include" / "heatcg.h", CSRC / "common.cuh", CSRC / "heat_common.cuh", CSRC / "tma.cuh",
           CSRC / "cg_common.cuh", CSRC / "xsum.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr"]


def nvcc_path() -> str:
    for cand in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if cand and (Path(cand) / "bin" / "nvcc").exists():
            return str(Path(cand) / "bin" / "nvcc")
    found = shutil.which("nvcc")
    if not found:
        raise RuntimeError("nvcc not found: set CUDA_HOME")
    return found


def _stale(target: Path, deps) -> bool:
    if not target.exists():
        return True
    t = target.stat().st_mtime
    return any(Path(d).stat().st_mtime > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> Path:
    BUILD.mkdir(exist_ok=True)
    nvcc = nvcc_path()
    inc = ["-I", str(ROOT / "include"), "-I", str(CSRC)]

    def compile_one(src: str) -> Path:
        obj = BUILD / (Path(src).stem + ".o")
        if force or _stale(obj, [CSRC / src] + HEADERS):
            cmd = [nvcc] + ARCH + NVCC_FLAGS + inc + ["-c", str(CSRC / src), "-o", str(obj)]
            if verbose:
                print(" ".join(cmd))
            subprocess.run(cmd, check=True)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    if force or _stale(LIB, objs):
        tmp = LIB.with_suffix(f".{os.getpid()}.tmp")
        cmd = [nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", str(tmp)] + [str(o) for o in objs]
        if verbose:
            print(" ".join(cmd))
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
