"""In-tree build of the native parts of the package.

* ``libqrsynth.so`` -- seeded input generators (plain C, host only).
* ``libquadrank.so`` -- the CUDA path (sm_103a kernels + C-ABI), compiled with
  nvcc, one translation unit per ``csrc/*.cu`` file, in parallel, then linked.

Nothing here is imported by the query path; the binding only loads the built
libraries and fails loudly if they are missing.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
CSRC = PKG / "csrc"
INCLUDE = PKG.parent / "include"
LIBDIR = PKG / "_lib"
SYNTH_SO = PKG / "synth" / "libqrsynth.so"
QR_SO = LIBDIR / "libquadrank.so"

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-Xptxas", "-warn-spills"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libquadrank.so")
    return cand


def _run(cmd: list[str]) -> None:
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"build step failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")


def _stale(target: Path, sources: list[Path]) -> bool:
    if not target.exists():
        return True
    t = target.stat().st_mtime
    return any(s.stat().st_mtime > t for s in sources)


def build_synth(force: bool = False) -> Path:
    src = PKG / "synth" / "synth.c"
    if force or _stale(SYNTH_SO, [src]):
        _run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", str(src), "-o", str(SYNTH_SO)])
    return SYNTH_SO


def build_cuda(force: bool = False, verbose_ptxas: bool = False) -> Path:
    cu = sorted(CSRC.glob("*.cu"))
    hdr = sorted(CSRC.glob("*.cuh")) + sorted(CSRC.glob("*.h")) + sorted(INCLUDE.glob("*.h"))
    cpp = sorted(CSRC.glob("*.cpp"))
    if not force and not _stale(QR_SO, cu + hdr + cpp):
        return QR_SO
    LIBDIR.mkdir(exist_ok=True)
    objdir = LIBDIR / "obj"
    objdir.mkdir(exist_ok=True)
    nvcc = _nvcc()
    inc = ["-I", str(INCLUDE), "-I", str(CSRC)]
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []

    def compile_one(src: Path) -> Path:
        obj = objdir / (src.name + ".o")
        if src.suffix == ".cu":
            _run([nvcc, *ARCH, *NVCC_FLAGS, *extra, *inc, "-c", str(src), "-o", str(obj)])
        else:
            _run(["g++", "-O2", "-std=c++17", "-fPIC", "-pthread", *inc,
                  "-I", "/usr/local/cuda/include", "-c", str(src), "-o", str(obj)])
        return obj

    with ThreadPoolExecutor(max_workers=max(1, min(len(cu) + len(cpp), os.cpu_count() or 4))) as ex:
        objs = list(ex.map(compile_one, cu + cpp))
    # static CUDA runtime: the library loads (and reports a clean error) on hosts without a driver
    _run([nvcc, *ARCH, "-shared", "-cudart", "static", "-o", str(QR_SO), *map(str, objs), "-lpthread"])
    return QR_SO


def build_all(force: bool = False) -> None:
    build_synth(force)
    build_cuda(force)
