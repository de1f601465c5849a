"""Build the CUDA library in-tree for sm_103a.

Each translation unit is compiled in parallel with nvcc, then linked into
``paper_2606_16765_gb300/lib/liblbm.so``.  Objects go to ``_build/`` (ignored
by git).  A unit is rebuilt when it or any header is newer than its object.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OBJ = os.path.join(ROOT, "_build")
LIBDIR = os.path.join(PKG, "lib")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-I" + os.path.join(ROOT, "include")] + ARCH

LIBS = {
    "liblbm.so": ["lbm_api.cu", "lbm_aux.cu", "lbm_step_f64.cu", "lbm_step_f32.cu",
                  "lbm_step_f16.cu", "lbm_step_bf16.cu", "lbm_step_f16c.cu", "lbm_noalloc.cu",
                  "resample.cu"],
    "libfno.so": ["fno.cu", "fno_umma.cu"],
    "libunet.so": ["unet.cu", "unet_gemm.cu"],
    "libffno.so": ["ffno.cu"],
}


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")
    return path


def _headers():
    return glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(ROOT, "include", "*.h"))


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src: str, extra) -> str:
    obj = os.path.join(OBJ, os.path.basename(src) + ".o")
    if _stale(obj, [src] + _headers() + [__file__]):
        tmp = obj + f".tmp{os.getpid()}"
        cmd = [nvcc()] + NVCC_FLAGS + list(extra) + ["-c", src, "-o", tmp]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        os.replace(tmp, obj)
    return obj


def build(verbose: bool = False, extra=()) -> dict:
    os.makedirs(OBJ, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    out = {}
    srcs = sorted({s for v in LIBS.values() for s in v})
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        objs = dict(zip(srcs, ex.map(lambda s: _compile(os.path.join(CSRC, s), extra), srcs)))
    for lib, units in LIBS.items():
        target = os.path.join(LIBDIR, lib)
        deps = [objs[u] for u in units]
        if _stale(target, deps):
            tmp = target + f".tmp{os.getpid()}"
            cmd = [nvcc(), "-shared", "-o", tmp] + deps + ARCH
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"link failed for {lib}:\n{r.stderr}")
            os.replace(tmp, target)
        out[lib] = target
        if verbose:
            print(target)
    return out


if __name__ == "__main__":
    build(verbose=True)
