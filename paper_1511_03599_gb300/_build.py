"""Build the in-tree CUDA library ``libppf.so`` for sm_103a with nvcc.

Every translation unit is compiled in parallel (the forward kernel once per
channel count C), then linked into one shared library beside this file.
Objects go to ``_build/`` (git-ignored).  Usage: ``python -m
paper_1511_03599_gb300._build`` or ``build()`` from Python.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUTDIR = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libppf.so")
CHANNELS = (32, 64, 128, 256, 512, 1024, 2048, 4096, 384, 768, 1536, 3072)
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags():
    return [ARCH, "-lineinfo", "-O3", "-std=c++17", "--expt-relaxed-constexpr",
            "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]


def _units():
    """(source, object, extra flags) for every translation unit."""
    units = []
    for src in sorted(glob.glob(os.path.join(CSRC, "*.cu"))):
        name = os.path.splitext(os.path.basename(src))[0]
        if name.endswith("_inst"):
            for C in CHANNELS:
                units.append((src, os.path.join(OUTDIR, f"{name}_c{C}.o"), [f"-DPPF_C={C}"]))
        else:
            units.append((src, os.path.join(OUTDIR, f"{name}.o"), []))
    return units


def _deps_mtime():
    files = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))
    return max((os.path.getmtime(f) for f in files), default=0.0)


def _compile(unit, force):
    src, obj, extra = unit
    newest = max(os.path.getmtime(src), _deps_mtime(), os.path.getmtime(__file__))
    if not force and os.path.exists(obj) and os.path.getmtime(obj) >= newest:
        return obj, None
    cmd = [nvcc()] + _flags() + extra + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        return obj, f"$ {' '.join(cmd)}\n{r.stdout}\n{r.stderr}"
    return obj, None


def build(force: bool = False, jobs: int | None = None, verbose: bool = False) -> str:
    """Compile and link; returns the path of libppf.so.  Raises on any error."""
    os.makedirs(OUTDIR, exist_ok=True)
    units = _units()
    jobs = jobs or max(1, min(len(units), os.cpu_count() or 1))
    errors = []
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        for obj, err in ex.map(lambda u: _compile(u, force), units):
            if err:
                errors.append(err)
            elif verbose:
                print("built", os.path.basename(obj))
    if errors:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
    objs = [u[1] for u in units]
    newest = max(os.path.getmtime(o) for o in objs)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < newest:
        tmp = LIB + ".tmp"
        cmd = [nvcc(), ARCH, "-shared", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n$ {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
