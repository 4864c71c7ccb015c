"""Build the native parts of the package in-tree.

* ``libmorph.so``  — the CUDA library behind ``include/morph.h`` (sm_103a only);
* ``libsynth.so``  — the seeded page generator (host C).

Compilation units are compiled in parallel; nothing is installed outside the
package directory.  ``python -m paper_0712_0121_gb300.build`` runs it.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")

CUDA_SOURCES = ["abi.cu", "packed.cu", "rle.cu", "batch.cu", "mask.cu", "noalloc.cu", "cc.cu", "transpose.cu", "skew.cu", "layout.cu",
                "rect.cu", "rect_k1w2.cu", "rect_k1w4.cu", "rect_k2w2.cu", "rect_k2w4.cu",
                "rle_rect_w2.cu", "rle_rect_w4.cu", "rle_mask.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-fvisibility=hidden",
              "-I" + INCLUDE, "-I" + CSRC]

LIBMORPH = os.path.join(PKG, "libmorph.so")
LIBSYNTH = os.path.join(PKG, "libsynth.so")


def nvcc() -> str:
    exe = shutil.which("nvcc")
    if exe:
        return exe
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found")


def _newer(target: str, deps) -> bool:
    if not os.path.exists(target):
        return False
    t = os.path.getmtime(target)
    return all(os.path.getmtime(d) <= t for d in deps)


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("command failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
    return r.stdout + r.stderr


def _deps():
    hdrs = [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    hdrs += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")]
    return hdrs


def build_morph(force: bool = False, verbose: bool = False, extra=()) -> str:
    os.makedirs(BUILD, exist_ok=True)
    srcs = [os.path.join(CSRC, s) for s in CUDA_SOURCES]
    if not force and _newer(LIBMORPH, srcs + _deps()):
        return LIBMORPH
    exe = nvcc()
    objs = [os.path.join(BUILD, os.path.basename(s)[:-3] + ".o") for s in srcs]
    flags = NVCC_FLAGS + list(extra) + (["-Xptxas", "-v"] if verbose else [])

    def compile_one(pair):
        src, obj = pair
        return _run([exe] + ARCH + flags + ["-c", src, "-o", obj])

    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        logs = list(ex.map(compile_one, zip(srcs, objs)))
    if verbose:
        for log in logs:
            sys.stdout.write(log)
    tmp = LIBMORPH + ".%d.tmp" % os.getpid()
    _run([exe] + ARCH + ["-shared", "-o", tmp] + objs)
    os.replace(tmp, LIBMORPH)
    return LIBMORPH


def build_synth(force: bool = False) -> str:
    src = os.path.join(CSRC, "synth.c")
    if not force and _newer(LIBSYNTH, [src]):
        return LIBSYNTH
    tmp = LIBSYNTH + ".%d.tmp" % os.getpid()
    # -ffp-contract=off: no fused multiply-add, so pages are identical on x86 and Arm hosts
    _run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fvisibility=hidden",
          "-o", tmp, src])
    os.replace(tmp, LIBSYNTH)
    return LIBSYNTH


def build_all(force: bool = False, verbose: bool = False) -> None:
    with cf.ThreadPoolExecutor(max_workers=2) as ex:
        f1 = ex.submit(build_morph, force, verbose)
        f2 = ex.submit(build_synth, force)
        f1.result()
        f2.result()


if __name__ == "__main__":
    build_all(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIBMORPH)
