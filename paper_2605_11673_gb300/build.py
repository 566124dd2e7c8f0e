"""In-tree build of libsta.so for sm_103a (nvcc, one -gencode, translation units in parallel).

    python -m paper_2605_11673_gb300.build [--force]

Output: paper_2605_11673_gb300/_build/libsta.so (git-ignored).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
CSRC = PKG / "csrc"
OUT = PKG / "_build"
LIB = OUT / "libsta.so"
INCLUDE = PKG.parent / "include"

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# --fmad=false: no implicit FMA contraction; the fixed evaluation order of the element matrix
# names every fused multiply-add explicitly (__fma_rn), so results are reproducible.
NVFLAGS = ["-O3", "-lineinfo", "--fmad=false", "-std=c++17", "-Xcompiler", "-fPIC",
           "-Xcompiler", "-fno-strict-aliasing", f"-I{INCLUDE}"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and Path(cand).exists():
            return cand
    raise RuntimeError("nvcc not found (CUDA toolkit required to build libsta)")


def sources():
    return sorted(CSRC.glob("*.cu"))


def _stale() -> bool:
    if not LIB.exists():
        return True
    t = LIB.stat().st_mtime
    deps = list(sources()) + list(CSRC.glob("*.cuh")) + list(INCLUDE.glob("*.h")) + [Path(__file__)]
    return any(p.stat().st_mtime > t for p in deps)


def build(force: bool = False, verbose: bool = False, out: Path | None = None,
          defines: tuple = (), src: Path | None = None) -> Path:
    """Compile every translation unit (of `src`, default csrc/) and link libsta.so (into `out`,
    default _build/)."""
    lib = Path(out) / "libsta.so" if out else LIB
    if out is None and not force and not _stale():
        return LIB
    odir = lib.parent
    odir.mkdir(parents=True, exist_ok=True)
    cc = nvcc()
    extra = [f"-D{d}" for d in defines]

    def compile_one(src: Path) -> Path:
        obj = odir / (src.stem + ".o")
        cmd = [cc, *ARCH, *NVFLAGS, *extra, "-c", str(src), "-o", str(obj)]
        if verbose:
            cmd.append("-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src.name}:\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, sorted(Path(src).glob("*.cu")) if src else sources()))
    tmp = lib.with_suffix(f".so.{os.getpid()}.tmp")
    r = subprocess.run([cc, *ARCH, "-shared", "-o", str(tmp), *map(str, objs)],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
