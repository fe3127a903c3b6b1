"""Build libaa_gb300.so (sm_103a only) in-tree, next to this file.

    python -m paper_1912_07704_gb300.build [--force] [--verbose]

Each translation unit under csrc/ is compiled by its own nvcc process (in
parallel); objects go to _build/ at the repository root.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OBJDIR = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libaa_gb300.so")
SOURCES = ["aa_plan.cpp", "aa_api.cpp", "aa_api_f32.cpp", "aa_profile.cpp", "aa_dedisp.cu",
           "aa_sps.cu", "aa_noalloc.cu", "aa_adjoint.cu", "aa_batch.cpp", "aa_autotune.cpp",
           "aa_server.cpp", "aa_fil.cpp", "aa_corner.cu", "aa_post.cu", "aa_subband.cu",
           "aa_pipeline.cpp", "aa_fused.cpp", "aa_fdmt.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libaa_gb300.so")
    return cand


def _flags(src: str, verbose: bool) -> list:
    f = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off,-O2",
         "-I", INCLUDE, "-I", CSRC]
    if src.endswith(".cu"):
        f += ARCH
        if verbose:
            f += ["-Xptxas", "-v"]
    else:
        f += ["-x", "cu"] + ARCH  # host-only TU, still through nvcc for the CUDA headers
    return f


def _deps() -> list:
    files = [os.path.join(CSRC, s) for s in SOURCES]
    files += [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith(".h")]
    files.append(os.path.join(INCLUDE, "aa_dedisp.h"))
    return files


def _stale(target: str, deps: list) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src: str, verbose: bool) -> tuple:
    obj = os.path.join(OBJDIR, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), "-c", os.path.join(CSRC, src), "-o", obj] + _flags(src, verbose)
    p = subprocess.run(cmd, capture_output=True, text=True)
    return src, obj, p.returncode, p.stdout + p.stderr


def build(force: bool = False, verbose: bool = False) -> str:
    deps = _deps()
    if not force and not _stale(LIB, deps):
        return LIB
    os.makedirs(OBJDIR, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose), SOURCES))
    failed = [r for r in results if r[2] != 0]
    for src, _, rc, out in results:
        if out.strip() and (verbose or rc != 0):
            sys.stderr.write(f"--- {src}\n{out}\n")
    if failed:
        raise RuntimeError("nvcc failed for " + ", ".join(r[0] for r in failed))
    tmp = LIB + ".tmp"
    cmd = [nvcc(), "-shared", "-o", tmp] + [r[1] for r in results] + ARCH + ["-lcuda"]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError("link failed:\n" + p.stdout + p.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--verbose", action="store_true")
    a = ap.parse_args()
    print(build(force=a.force, verbose=a.verbose))
