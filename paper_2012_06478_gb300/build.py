"""Build the engine's shared library (librms.so) in-tree with nvcc for sm_103a.

The plain FP64 form and the C-ABI/set-up/read-out unit are compiled with
-fmad=false (no FMA contraction, so every operation rounds as in the CPU
reference); the FP32 forms keep FMA contraction.  The translation units
compile in parallel; the link uses nvcc's static CUDA runtime.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "librms.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
          "--expt-relaxed-constexpr"]
UNITS = [("rms_api.cu", ["-fmad=false", "-Xcompiler", "-ffp-contract=off"]), ("walk_fp64.cu", ["-fmad=false"]), ("walk_fp32.cu", ["-fmad=true"]),
         ("walk_reject_fp64.cu", ["-fmad=false"]), ("walk_reject_fp32.cu", ["-fmad=true"]),
         ("walk_mt_fp64.cu", ["-fmad=false"]), ("walk_mt_fp32.cu", ["-fmad=true"]),
         ("rms_noalloc.cu", ["-fmad=false"]), ("rms_morton.cu", []), ("rms_serve.cu", ["-fmad=false"]), ("rms_peaks.cu", ["-fmad=false"])]


def _sources():
    inc = os.path.join(ROOT, "include")
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h"))] + \
        [os.path.join(inc, f) for f in os.listdir(inc) if f.endswith(".h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = os.environ.get("NVCC", "nvcc")
    procs = []
    objs = []
    for src, extra in UNITS:
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *COMMON, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        if ptxas_info:
            cmd.insert(1, "-Xptxas=-v")
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
        objs.append(obj)
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append(f"{src}:\n{out}")
        elif out and (verbose or ptxas_info):
            print(out, file=sys.stderr)
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(failed))
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call([nvcc, *ARCH, "-shared", "-o", tmp, *objs])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
