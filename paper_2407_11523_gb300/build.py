"""Build libbpq.so in-tree with nvcc for sm_103a (GB300).

Each translation unit is compiled in parallel into _build/, then linked into
paper_2407_11523_gb300/libbpq.so.  Run `python -m paper_2407_11523_gb300.build`
or call build().
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libbpq.so")
BUILD_DIR = os.path.join(HERE, "_build")
SOURCES = ["api.cu", "batch.cu", "server.cu", "train.cu", "decode.cu", "decode_plain.cu", "decode_momentum.cu", "decode_adagrad.cu",
           "decode_ewainit.cu", "decode_aewa.cu", "decode_plain_full.cu", "decode_momentum_full.cu",
           "decode_adagrad_full.cu", "decode_ewainit_full.cu", "decode_aewa_full.cu", "decode_plain_pair.cu",
           "decode_momentum_pair.cu", "decode_adagrad_pair.cu", "decode_ewainit_pair.cu", "decode_plain_batch.cu",
           "decode_momentum_batch.cu", "decode_adagrad_batch.cu", "decode_ewainit_batch.cu", "serve_kernels.cu",
           "decode_debug.cu", "serial.cu", "serial_pair.cu", "tanner.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale() -> bool:
    if not os.path.exists(OUT):
        return True
    t = os.path.getmtime(OUT)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(HERE, "..", "include", "bpq.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    if not force and not _stale():
        return OUT
    os.makedirs(BUILD_DIR, exist_ok=True)
    cc = nvcc()
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", *ARCH, *extra_flags]
    procs = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(BUILD_DIR, src + ".o")
        objs.append(obj)
        cmd = [cc, *common, "-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cu") and verbose:
            cmd += ["-Xptxas", "-v"]
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode:
            failed.append(src)
    if failed:
        raise RuntimeError(f"nvcc failed on {failed}")
    tmp = OUT + f".tmp{os.getpid()}"
    subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs], check=True)
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(OUT)
