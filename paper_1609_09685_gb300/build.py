"""Build the CUDA library in-tree for sm_103a with nvcc (no cmake).

``python -m paper_1609_09685_gb300.build`` compiles each ``csrc/*.cu`` to an
object in parallel and links ``_lib/liblbm_gb300.so``.  The same commands work
on x86_64 and aarch64 hosts (nvcc cross-compiles device code without a GPU).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
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
LIB = os.path.join(LIBDIR, "liblbm_gb300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def kernel_hash() -> str:
    """Hash of the CUDA sources and the C header: the autotuner's cache key
    carries it, so a cached launch configuration is dropped when a kernel
    changes."""
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(CSRC, "*.cu*")) + glob.glob(os.path.join(CSRC, "*.h")) +
                    [os.path.join(INCLUDE, "lbm.h")]):
        with open(f, "rb") as fh:
            h.update(os.path.basename(f).encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def _flags(defines=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "-I", INCLUDE, "-I", CSRC, f'-DLBM_KERNEL_HASH="{kernel_hash()}"'] + [f"-D{d}" for d in defines]


def _stamp(srcs, defines=()):
    h = hashlib.sha256()
    for f in sorted(srcs + glob.glob(os.path.join(CSRC, "*.h*")) + [os.path.join(INCLUDE, "lbm.h")]):
        with open(f, "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    h.update(" ".join(_flags(defines)).encode())
    h.update(os.uname().machine.encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, defines=(), out: str = None) -> str:
    """Compile and link the library; `defines` are extra -D tuning macros and
    `out` an alternative output path (both for tuning sweeps)."""
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    lib = out or LIB
    libdir = os.path.dirname(lib)
    os.makedirs(libdir, exist_ok=True)
    stamp_file = lib + ".stamp"
    stamp = _stamp(srcs, defines)
    if not force and os.path.exists(lib) and os.path.exists(stamp_file):
        with open(stamp_file) as fh:
            if fh.read().strip() == stamp:
                return lib
    cc = nvcc()
    tag = hashlib.sha256(lib.encode()).hexdigest()[:8]
    objs = [os.path.join(libdir, os.path.basename(s)[:-3] + f".{tag}.o") for s in srcs]

    def compile_one(src_obj):
        src, obj = src_obj
        cmd = [cc] + _flags(defines) + ["-c", src, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        logs = list(ex.map(compile_one, zip(srcs, objs)))
    if verbose:
        for l in logs:
            sys.stderr.write(l)
    tmp = lib + f".tmp{os.getpid()}"
    r = subprocess.run([cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    with open(stamp_file, "w") as fh:
        fh.write(stamp)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
