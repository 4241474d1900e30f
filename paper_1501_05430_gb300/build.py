"""Build liblbm.so (the C-ABI library) in-tree with nvcc for sm_103a.

Translation units and their floating-point flags:
  lbm_ref.cu, lbm_measure.cu,  -fmad=false: the canonical-order kernels must not
  lbm_adjoint.cu               contract a*b+c into an FMA (bit-exact FP64 path;
                               the adjoint recomputes the same forward values)
  lbm_fused.cu, lbm_batch.cu   FMA allowed: the production FP32 step (one domain; many
                               instances in one persistent launch)
  lbm_api.cu                   host code and launch orchestration
Units compile in parallel; only stale objects are rebuilt.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "liblbm.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
UNITS = {
    "lbm_api.cu": [],
    "lbm_ref.cu": ["-fmad=false"],
    "lbm_measure.cu": ["-fmad=false"],
    "lbm_fused.cu": [],
    "lbm_noalloc.cu": [],
    "lbm_batch.cu": [],
    "lbm_adjoint.cu": ["-fmad=false"],
}
HEADERS = [os.path.join(CSRC, h) for h in ("lbm_internal.h", "lbm_node.cuh", "lbm_ref_node.cuh")] + [
    os.path.join(ROOT, "include", "lbm.h")]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every unit that changed and link liblbm.so; return its path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
                     "-I", os.path.join(ROOT, "include"), "-I", CSRC]
    procs, objs = [], []
    for src, extra in UNITS.items():
        path = os.path.join(CSRC, src)
        obj = os.path.join(OUT_DIR, src.replace(".cu", ".o"))
        objs.append(obj)
        if force or _stale(obj, [path] + HEADERS):
            cmd = [nvcc] + common + extra + ["-c", path, "-o", obj]
            if verbose:
                print(" ".join(cmd), flush=True)
            procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((cmd, out.decode(errors="replace")))
        elif verbose and out:
            print(out.decode(errors="replace"), flush=True)
    if failed:
        msg = "\n".join(f"$ {' '.join(c)}\n{o}" for c, o in failed)
        raise RuntimeError(f"nvcc failed:\n{msg}")
    if force or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
