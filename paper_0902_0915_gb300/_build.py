"""Build of libmwax.so: every CUDA source of the package compiled for sm_103a
with nvcc (in parallel), linked into one shared library inside the package."""
from __future__ import annotations

import glob
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "_lib", "libmwax.so")
ARCH = "sm_103a"


def nvcc_flags() -> list[str]:
    comp = ARCH.replace("sm_", "compute_")
    return ["-gencode", f"arch={comp},code={ARCH}", "-O3", "-lineinfo", "-std=c++17",
            "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link; returns the library path."""
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    objs, cmds = [], []
    for src in sources():
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        objs.append(obj)
        cmds.append(["nvcc", *nvcc_flags(), "-c", src, "-o", obj])

    def run(c):
        return subprocess.run(c, capture_output=True, text=True)

    with ThreadPoolExecutor(max(1, min(len(cmds), os.cpu_count() or 1))) as ex:
        results = list(ex.map(run, cmds))
    for c, r in zip(cmds, results):
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed: {' '.join(c)}\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
    tmp = LIB + ".tmp"
    link = ["nvcc", "-gencode", f"arch={ARCH.replace('sm_', 'compute_')},code={ARCH}", "-shared",
            *objs, "-o", tmp]
    r = run(link)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(link)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB
