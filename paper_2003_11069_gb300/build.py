"""Build the CUDA library liblbnci.so (sm_103a) in-tree with nvcc.

The translation units compile in parallel; the FP64 one is built with --fmad=false
(no multiply-add contraction). Output: paper_2003_11069_gb300/_lib/liblbnci.so.
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "liblbnci.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

UNITS = {
    "lb_api.cu": [],
    "lb_fp64.cu": ["--fmad=false"],
    "lb_fp32.cu": [],
    "lb_tma2d.cu": [],
    "lb_carry3d.cu": [],
    "lb_fp16.cu": [],
    "unet_api.cu": [],
}


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbnci.so")


def _cuda_libdir(nvcc: str) -> str:
    root = os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    for sub in ("lib64", "lib", "targets/sbsa-linux/lib", "targets/x86_64-linux/lib"):
        d = os.path.join(root, sub)
        if os.path.exists(os.path.join(d, "libcudart.so")):
            return d
    return os.path.join(root, "lib64")


def _sources_digest() -> str:
    h = hashlib.sha256()
    for d in (CSRC, INCLUDE):
        for name in sorted(os.listdir(d)):
            with open(os.path.join(d, name), "rb") as fh:
                h.update(name.encode())
                h.update(fh.read())
    h.update(" ".join(ARCH).encode())
    h.update(repr(sorted(UNITS.items())).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile and link liblbnci.so; skipped when the sources are unchanged."""
    os.makedirs(LIBDIR, exist_ok=True)
    stamp = os.path.join(LIBDIR, "liblbnci.sha256")
    digest = _sources_digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as fh:
            if fh.read().strip() == digest:
                return LIB
    nvcc = _nvcc()
    objdir = os.path.join(LIBDIR, "obj")
    os.makedirs(objdir, exist_ok=True)
    common = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE]
    if ptxas_info:
        common += ["-Xptxas", "-v"]
    procs = []
    for unit, extra in UNITS.items():
        obj = os.path.join(objdir, unit.replace(".cu", ".o"))
        cmd = [nvcc, "-c", os.path.join(CSRC, unit), "-o", obj] + common + extra
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((unit, obj, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    objs, errors = [], []
    for unit, obj, pr in procs:
        out, _ = pr.communicate()
        if pr.returncode != 0:
            errors.append(f"{unit}:\n{out.decode(errors='replace')}")
        elif verbose or ptxas_info:
            sys.stderr.write(out.decode(errors="replace"))
        objs.append(obj)
    if errors:
        raise RuntimeError("nvcc failed\n" + "\n".join(errors))
    tmp = LIB + f".tmp{os.getpid()}"
    link = [nvcc, "-shared", "-o", tmp] + objs + ARCH + [
        "-cudart", "shared", "-Xlinker", "-rpath," + _cuda_libdir(nvcc)]
    subprocess.run(link, check=True)
    os.replace(tmp, LIB)
    with open(stamp, "w") as fh:
        fh.write(digest)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
