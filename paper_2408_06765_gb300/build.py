"""Build librsi.so (the sm_103a CUDA library behind include/rsi.h) in-tree.

    python -m paper_2408_06765_gb300.build [--force]

Each .cu file is compiled by nvcc in parallel for sm_103a only, then linked
into paper_2408_06765_gb300/_build/librsi.so (static CUDA runtime).  ptxas
resource usage (-Xptxas -v) is kept in _build/ptxas.log.  RSI_BUILD_DEFINES
(-D flags for the kernels' tuning knobs) builds into _build_<hash> instead,
and the binding loads that library.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import platform
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")


def extra_defines() -> list:
    """Build-time tuning defines from RSI_BUILD_DEFINES (e.g.
    "-DRSI_FP32_PACKED_RSI_MIN_BLOCKS=3"); only -D flags are accepted."""
    toks = os.environ.get("RSI_BUILD_DEFINES", "").split()
    for t in toks:
        if not t.startswith("-D"):
            raise ValueError(f"RSI_BUILD_DEFINES takes -D flags only, got {t!r}")
    return toks


def build_dir() -> str:
    """_build, or _build_<hash> for a build with extra defines."""
    d = extra_defines()
    if not d:
        return os.path.join(HERE, "_build")
    import hashlib
    return os.path.join(HERE, "_build_" + hashlib.sha256(" ".join(d).encode()).hexdigest()[:12])


BUILD = build_dir()
LIB = os.path.join(BUILD, "librsi.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xptxas", "-v",
          "--expt-relaxed-constexpr"]


def nvcc() -> str:
    cand = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the RSI CUDA library cannot be built")
    return cand


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _deps():
    inc = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]  # any header
    inc.append(os.path.join(os.path.dirname(HERE), "include", "rsi.h"))
    return inc


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in [src] + _deps())


def _compile(src: str, force: bool):
    obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
    if not force and not _stale(obj, src):
        return obj, ""
    cmd = [nvcc()] + ARCH + CFLAGS + extra_defines() + ["-c", src, "-o", obj + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
    os.replace(obj + ".tmp", obj)
    return obj, r.stdout + r.stderr


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    stamp = os.path.join(BUILD, "machine.txt")
    here = platform.machine()
    if not os.path.exists(stamp) or open(stamp).read().strip() != here:
        force = True  # objects from another host architecture are never reused
    srcs = sources()
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        results = list(ex.map(lambda s: _compile(s, force), srcs))
    logs = [log for _, log in results if log]
    if logs:
        with open(os.path.join(BUILD, "ptxas.log"), "w") as f:
            f.write("\n".join(logs))
    objs = [o for o, _ in results]
    if force or not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(here)
    if verbose:
        print(LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
