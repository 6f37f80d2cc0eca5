"""Build libsdcsz.so in-tree with nvcc for sm_103a (GB300).

Each CUDA translation unit compiles in parallel to an object file under ``_build/``, then the
objects link into ``libsdcsz.so`` next to this file. IEEE arithmetic is required by the
compressor's bit-exact contract: no FMA contraction, IEEE division and square root, no
flush-to-zero.
"""

from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libsdcsz.so")
# measurement helper (FP64 instruction rate), kept out of the compressor's library
PEAK_SRC = "peak_fp64.cu"
PEAK_LIB = os.path.join(HERE, "libsdcsz_peak.so")
SOURCES = ["api.cu", "k_prep.cu", "k_predict_f32.cu", "k_predict_f64.cu", "k_predict_f32c.cu", "k_predict_f64c.cu",
           "k_flip.cu", "k_codebook.cu", "k_encode.cu", "k_decode_f32.cu", "k_decode_f64.cu", "k_decode_f32c.cu",
           "k_decode_f64c.cu", "k_decode_wave.cu", "k_lossless.cu", "server.cu", "shard.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-fmad=false", "-prec-div=true", "-prec-sqrt=true", "-ftz=false",
         "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the sdcsz CUDA library cannot be built")


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(INCLUDE, "sdcsz.h"))
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        if force or _stale(o, [s] + headers):
            jobs.append([nvcc, *ARCH, *FLAGS, *extra_flags, "-c", s, "-o", o])

    def run(cmd):
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr, file=sys.stderr)

    lib_jobs = len(jobs)
    peak_src = os.path.join(CSRC, PEAK_SRC)
    if force or _stale(PEAK_LIB, [peak_src]):
        jobs.append([nvcc, *ARCH, *FLAGS, *extra_flags, "-shared", peak_src, "-o", PEAK_LIB])
    with cf.ThreadPoolExecutor(max_workers=len(jobs) or 1) as ex:
        list(ex.map(run, jobs))
    objs = [os.path.join(BUILD, s.replace(".cu", ".o")) for s in SOURCES]
    if force or lib_jobs or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        run([nvcc, *ARCH, "-shared", "-o", tmp, *objs])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
