"""In-tree build of the package's native parts.

* ``libsda.so``   - the C-ABI library (CUDA kernels for sm_103a + host runtime),
                     built with nvcc from ``csrc/``.
* ``_synth_native.so`` - the input generator's native helpers (kNN graph, large
                     workloads), built with gcc.

Everything is compiled in place next to its sources; nothing is installed.
"""
from __future__ import annotations

import os
import platform
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG_DIR = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG_DIR, "csrc")
LIBSDA = os.path.join(PKG_DIR, "libsda.so")
SYNTH_SO = os.path.join(PKG_DIR, "_synth_native.so")
MACHINE = platform.machine()
BUILD_DIR = os.path.join(PKG_DIR, "_build", MACHINE)

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _newer(target: str, sources: list[str]) -> bool:
    """True if `target` is missing, older than a source, or built for another machine."""
    if not os.path.exists(target):
        return True
    stamp = target + ".arch"
    if not os.path.exists(stamp) or open(stamp).read().strip() != MACHINE:
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in sources)


def _stamp(target: str) -> None:
    with open(target + ".arch", "w") as f:
        f.write(MACHINE + "\n")


def _run(cmd: list[str]) -> None:
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)


def build_synth(force: bool = False) -> str:
    src = os.path.join(PKG_DIR, "synth_native.c")
    if force or _newer(SYNTH_SO, [src]):
        tmp = SYNTH_SO + ".tmp%d" % os.getpid()
        _run(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", src, "-o", tmp, "-lm"])
        os.replace(tmp, SYNTH_SO)
        _stamp(SYNTH_SO)
    return SYNTH_SO


def _cuda_sources() -> tuple[list[str], list[str]]:
    cu = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))
    hdr = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h")))
    hdr.append(os.path.join(os.path.dirname(PKG_DIR), "include", "sda.h"))
    return cu, hdr


def build_libsda(force: bool = False, verbose_ptxas: bool = False) -> str:
    cu, hdr = _cuda_sources()
    if not (force or _newer(LIBSDA, cu + hdr)):
        return LIBSDA
    os.makedirs(BUILD_DIR, exist_ok=True)
    inc = ["-I", os.path.join(os.path.dirname(PKG_DIR), "include"), "-I", CSRC]
    common = ARCH_FLAGS + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                           "-Xcompiler", "-fvisibility=hidden", "--expt-relaxed-constexpr"] + inc
    if verbose_ptxas:
        common += ["-Xptxas", "-v"]
    objs = []

    def compile_one(src: str) -> str:
        obj = os.path.join(BUILD_DIR, os.path.basename(src) + ".o")
        if force or _newer(obj, [src] + hdr):
            _run([NVCC] + common + ["-c", src, "-o", obj])
            _stamp(obj)
        return obj

    with ThreadPoolExecutor(max_workers=min(8, len(cu))) as ex:
        objs = list(ex.map(compile_one, cu))
    tmp = LIBSDA + ".tmp%d" % os.getpid()
    _run([NVCC] + ARCH_FLAGS + ["-shared", "-o", tmp] + objs)
    os.replace(tmp, LIBSDA)
    _stamp(LIBSDA)
    return LIBSDA


def build_all(force: bool = False) -> None:
    build_synth(force)
    build_libsda(force)


if __name__ == "__main__":
    build_all(force="--force" in sys.argv)
    print(LIBSDA)
