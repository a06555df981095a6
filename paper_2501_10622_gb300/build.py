"""Builds libcwthf.so in-tree from csrc/*.cu for sm_103a (nvcc, no cmake).

Each translation unit is compiled in parallel, then linked into one shared
library with the CUDA runtime linked statically.  The library exports only
the C ABI declared in include/cwthf.h.  build(checked=True) builds the same
sources with CWTHF_CHECKED defined into libcwthf_checked.so (device-side
range checks of data-driven indices; the binding loads it when the
environment sets CWTHF_CHECKED=1).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
OUT = PKG / "libcwthf.so"
OUT_CHECKED = PKG / "libcwthf_checked.so"
BUILD = ROOT / "_build"
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and Path(cand).exists():
            return cand
    raise RuntimeError("nvcc not found")


def flags(extra=()):
    return [ARCH, "-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
            "-Xcompiler", "-fvisibility=hidden", f"-I{ROOT / 'include'}", *extra]


def sources():
    return sorted(CSRC.glob("*.cu"))


def _stale(target: Path, deps) -> bool:
    if not target.exists():
        return True
    t = target.stat().st_mtime
    return any(d.stat().st_mtime > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, checked: bool = False) -> Path:
    out = OUT_CHECKED if checked else OUT
    bdir = BUILD / "checked" if checked else BUILD
    bdir.mkdir(parents=True, exist_ok=True)
    headers = list(CSRC.glob("*.cuh")) + [ROOT / "include" / "cwthf.h"]
    srcs = sources()
    objs = [bdir / (s.stem + ".o") for s in srcs]
    extra = (["-Xptxas", "-v"] if ptxas_info else []) + (["-DCWTHF_CHECKED"] if checked else [])

    def compile_one(pair):
        src, obj = pair
        if not force and not ptxas_info and not _stale(obj, [src, *headers]):
            return ""
        cmd = [nvcc(), *flags(extra), "-c", str(src), "-o", str(obj)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src.name}:\n{r.stderr}")
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        logs = list(ex.map(compile_one, zip(srcs, objs)))
    if verbose or ptxas_info:
        for s, log in zip(srcs, logs):
            if log:
                print(f"--- {s.name}\n{log}")
    if force or _stale(out, objs):
        tmp = out.with_suffix(f".so.{os.getpid()}")
        cmd = [nvcc(), ARCH, "-shared", "-Xcompiler", "-fPIC", *map(str, objs), "-ldl", "-o", str(tmp)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, out)
    return out


def build_all(force: bool = False) -> list[Path]:
    """The library and its checked variant, compiled side by side."""
    with cf.ThreadPoolExecutor(max_workers=2) as ex:
        return list(ex.map(lambda c: build(force=force, checked=c), (False, True)))


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
