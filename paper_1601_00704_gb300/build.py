"""Compile the CUDA library libglbm.so in-tree for sm_103a with nvcc."""

from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = [os.path.join(HERE, "csrc", f) for f in ("glbm.cu", "batch.cu", "nn.cu", "nn_tc.cu", "nn_tc_train.cu", "em.cu")]
HDR = [os.path.join(HERE, "csrc", n) for n in ("glbm_kernels.cuh", "setup_kernels.cuh", "tc_common.cuh", "trace.h", "guard.h")]
OBJ = os.path.join(HERE, "csrc", "_obj")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libglbm.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libglbm")
    return exe


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = SRC + HDR + [os.path.join(INCLUDE, "glbm.h"), __file__]
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    """Build libglbm.so next to this file (skipped when up to date)."""
    if not force and not _stale():
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    os.makedirs(OBJ, exist_ok=True)
    flags = [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE]
    if verbose:
        flags.insert(0, "-Xptxas=-v")
    if extra:
        flags = list(extra) + flags
    procs, objs = [], []
    for src in SRC:
        obj = os.path.join(OBJ, os.path.basename(src) + f".{os.getpid()}.o")
        objs.append(obj)
        procs.append((src, subprocess.Popen([nvcc(), *flags, "-c", src, "-o", obj],
                                            stdout=subprocess.PIPE, stderr=subprocess.STDOUT,
                                            text=True)))
    log = ""
    failed = False
    for src, p in procs:
        out, _ = p.communicate()
        log += out
        failed = failed or p.returncode != 0
    if not failed:
        r = subprocess.run([nvcc(), *ARCH, "-shared", *objs, "-o", tmp],
                           capture_output=True, text=True)
        log += r.stdout + r.stderr
        failed = r.returncode != 0
    for o in objs:
        if os.path.exists(o):
            os.remove(o)
    if failed:
        raise RuntimeError("nvcc failed:\n" + log)
    if verbose:
        print(log)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
