"""Build libxy.so (the sm_103a kernels and the C ABI of include/xy.h) in-tree.

    python -m paper_1210_6116_b300.build
"""
from __future__ import annotations

import os
import subprocess
import sys
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
SRC = PKG / "csrc"
LIB = PKG / "libxy.so"
# the bounds-checked build (-DXY_BOUNDS_CHECK): data-derived global indices
# are tested on the device and reported as XY_EINTERNAL (the binding loads it
# when XY_BOUNDS_CHECK=1 is set in the environment)
LIB_CHECKED = PKG / "libxy_checked.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(SRC.glob("*.cu")) + sorted(SRC.glob("*.cuh")) + [ROOT / "include" / "xy.h"]


def needs_build(lib: Path = LIB) -> bool:
    if not lib.exists():
        return True
    t = lib.stat().st_mtime
    return any(p.stat().st_mtime > t for p in sources())


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> Path:
    """Compile the three translation units in parallel (one nvcc each), then
    link them into libxy.so (checked=True: the bounds-checked
    libxy_checked.so)."""
    lib = LIB_CHECKED if checked else LIB
    if not force and not needs_build(lib):
        return lib
    tmp = lib.with_suffix(f".so.tmp{os.getpid()}")
    flags = [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
             "-diag-suppress", "128", "-I", str(ROOT / "include")]
    if checked:
        flags.append("-DXY_BOUNDS_CHECK")
    if verbose:
        flags.insert(0, "-Xptxas=-v")
    objs, procs = [], []
    for name in ("xy_api.cu", "xy_engine.cu", "xy_static.cu"):
        obj = lib.parent / f".{name[:-3]}{'_checked' if checked else ''}.{os.getpid()}.o"
        objs.append(obj)
        procs.append(subprocess.Popen(["nvcc", *flags, "-c", str(SRC / name), "-o", str(obj)]))
    try:
        codes = [pr.wait() for pr in procs]
        if any(codes):
            raise subprocess.CalledProcessError(max(codes), "nvcc -c")
        subprocess.run(["nvcc", *ARCH, "-shared", *map(str, objs), "-o", str(tmp)], check=True)
    finally:
        for obj in objs:
            obj.unlink(missing_ok=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
