"""Build the in-tree CUDA libraries for sm_103a (GB300).

    python -m paper_1910_10063_gb300.build          # libskx.so + libskx_synth.so

Each .cu translation unit is compiled in parallel with
``nvcc -gencode arch=compute_103a,code=sm_103a -O3 -lineinfo`` and linked
into a shared library next to this file.  Rebuilds only what changed.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(PKG, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O3",
              "--expt-relaxed-constexpr", "-I", INCLUDE]

LIBS = {
    "libskx.so": {
        "dir": os.path.join(PKG, "csrc"),
        "sources": ["api.cu", "histogram.cu", "histogram_part.cu", "sort.cu", "remap.cu", "probe.cu", "probe_split.cu", "autotune.cu", "batch.cu", "server.cu", "operators.cu",
                    "cache_model.cu", "noalloc.cu"],
        "headers": ["skx_internal.cuh", "probe_core.cuh", os.path.join(INCLUDE, "skx.h")],
    },
    "libskx_synth.so": {
        "dir": os.path.join(PKG, "synth"),
        "sources": ["synth.cu"],
        "headers": [os.path.join(INCLUDE, "skx_synth.h")],
    },
}


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libskx")
    return path


def _mtime(p: str) -> float:
    return os.path.getmtime(p) if os.path.exists(p) else 0.0


def _compile(src: str, obj: str, deps: list[str], verbose: bool) -> str:
    newest = max(_mtime(d) for d in [src] + deps)
    if _mtime(obj) >= newest:
        return obj
    cmd = [nvcc()] + ARCH + NVCC_FLAGS + ["-c", src, "-o", obj + ".tmp"]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if verbose and r.stderr:
        sys.stderr.write(r.stderr)
    os.replace(obj + ".tmp", obj)
    return obj


def build(verbose: bool = False, jobs: int | None = None) -> dict[str, str]:
    os.makedirs(BUILD_DIR, exist_ok=True)
    tasks = []
    for lib, spec in LIBS.items():
        deps = [h if os.path.isabs(h) else os.path.join(spec["dir"], h) for h in spec["headers"]]
        for s in spec["sources"]:
            src = os.path.join(spec["dir"], s)
            obj = os.path.join(BUILD_DIR, lib.replace(".so", "") + "_" + s.replace(".cu", ".o"))
            tasks.append((lib, src, obj, deps))
    with ThreadPoolExecutor(max_workers=jobs or min(8, os.cpu_count() or 4)) as ex:
        futs = [(lib, ex.submit(_compile, src, obj, deps, verbose)) for lib, src, obj, deps in tasks]
        objs: dict[str, list[str]] = {}
        for lib, f in futs:
            objs.setdefault(lib, []).append(f.result())
    out = {}
    for lib, olist in objs.items():
        target = os.path.join(PKG, lib)
        if _mtime(target) < max(_mtime(o) for o in olist):
            tmp = target + f".tmp{os.getpid()}"
            cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + olist
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"link failed for {lib}:\n{r.stdout}\n{r.stderr}")
            os.replace(tmp, target)
        out[lib] = target
    return out


if __name__ == "__main__":
    for k, v in build(verbose="-v" in sys.argv).items():
        print(k, "->", v)
