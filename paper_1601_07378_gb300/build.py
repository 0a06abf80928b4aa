"""Build the sm_103a shared library libvloc.so in-tree (no cmake, no pip).

The translation units of ``csrc/`` (the compile-time-length FP32 and
double-float kernels split over three files each, one per precision for the
runtime-radix kernels, the dispatch, the plan and the no-alloc entry) are compiled in parallel with
nvcc and linked into ``paper_1601_07378_gb300/_build/libvloc.so``
against the shared CUDA runtime, so the library shares the runtime PyTorch
already loaded.  ``python -m paper_1601_07378_gb300.build`` rebuilds it.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libvloc.so")
ROOT = os.path.dirname(HERE)

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["kernels_ct_a.cu", "kernels_ct_b.cu", "kernels_ct_c.cu", "kernels_df_a.cu", "kernels_df_b.cu",
           "kernels_df_c.cu", "kernels_f32.cu", "kernels_f64.cu", "kernels.cu", "plan.cpp", "noalloc.cu", "peaks.cu"]


def _cuda_home() -> str:
    home = os.environ.get("CUDA_HOME") or os.environ.get("CUDA_PATH")
    if home and os.path.exists(os.path.join(home, "bin", "nvcc")):
        return home
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    return "/usr/local/cuda"


def _deps() -> list[str]:
    out = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    out.append(os.path.join(ROOT, "include", "vloc.h"))
    out.append(os.path.abspath(__file__))
    return out


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libvloc.so for sm_103a if it is missing or stale; return its path."""
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + os.path.join(ROOT, "include"), "-I" + CSRC]
    cu_flags = ARCH + ["-lineinfo", "--expt-relaxed-constexpr", "-Xptxas", "-warn-spills"]
    procs = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(BUILD, src + f".{os.getpid()}.o")
        cmd = [nvcc, *common]
        if src.endswith(".cu"):
            cmd += cu_flags
        else:
            cmd += ["-x", "c++"]
        cmd += ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        text = out.decode(errors="replace")
        if p.returncode != 0:
            failed.append(f"--- {src} ---\n{text}")
        elif verbose and text.strip():
            print(text, flush=True)
    if failed:
        raise RuntimeError("libvloc build failed:\n" + "\n".join(failed))
    tmp = LIB + f".{os.getpid()}.tmp"
    link = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
            "-Xlinker", "-rpath," + os.path.join(cuda, "lib64")]
    if verbose:
        print(" ".join(link), flush=True)
    subprocess.check_call(link)
    os.replace(tmp, LIB)
    for o in objs:
        try:
            os.remove(o)
        except OSError:
            pass
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
