"""In-tree build of the package's native libraries.

``liblbm_gb300.so``: the CUDA kernels and the C ABI, compiled by nvcc for
sm_103a only.  ``libgeom.so``: the seeded voxel-image generators (plain C).
Both land in ``paper_1902_11193_gb300/lib/``.
"""
from __future__ import annotations

import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIBDIR = os.path.join(PKG, "lib")
INCLUDE = os.path.join(ROOT, "include")

GEOM_SO = os.path.join(LIBDIR, "libgeom.so")
LBM_SO = os.path.join(LIBDIR, "liblbm_gb300.so")

CUDA_SOURCES = ["lbm_api.cu", "lbm_kernels.cu", "lbm_links.cu", "lbm_adjoint.cu", "lbm_batch.cu",
                "lbm_noalloc.cu", "lbm_domain.cu"]
CUDA_HEADERS = ["lbm_internal.cuh", "lbm_ctx.h", "lbm_collide.cuh", "lbm_sparse.cuh", "lbm_step.cuh"]
NVCC_ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    p = os.path.join(home, "bin", "nvcc")
    return p if os.path.exists(p) else "nvcc"


def _stale(out: str, deps: list[str]) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build_geometry(force: bool = False) -> str:
    src = os.path.join(CSRC, "geometry.c")
    if force or _stale(GEOM_SO, [src]):
        os.makedirs(LIBDIR, exist_ok=True)
        tmp = GEOM_SO + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-D_DEFAULT_SOURCE",
                        "-o", tmp, src, "-lm"], check=True)
        os.replace(tmp, GEOM_SO)
    return GEOM_SO


def build_lbm(force: bool = False, extra_flags: list[str] | None = None,
              out: str | None = None) -> str:
    """Builds liblbm_gb300.so (or, with `out`, a variant such as the
    bounds-check build, -DLBM_BOUNDS_CHECK, at that path, objects beside it)."""
    so = out or LBM_SO
    srcs = [os.path.join(CSRC, s) for s in CUDA_SOURCES]
    deps = srcs + [os.path.join(CSRC, h) for h in CUDA_HEADERS] + [os.path.join(INCLUDE, "lbm.h")]
    if not (force or _stale(so, deps)):
        return so
    os.makedirs(os.path.dirname(so), exist_ok=True)
    objdir = os.path.join(os.path.dirname(so), "obj")
    os.makedirs(objdir, exist_ok=True)
    flags = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", *NVCC_ARCH,
             "-I", INCLUDE, "-I", CSRC, "--expt-relaxed-constexpr", *(extra_flags or [])]

    def compile_one(src: str) -> str:
        obj = os.path.join(objdir, os.path.basename(src) + ".o")
        subprocess.run([_nvcc(), *flags, "-c", src, "-o", obj], check=True)
        return obj

    with ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = so + f".tmp{os.getpid()}"
    subprocess.run([_nvcc(), "-shared", *NVCC_ARCH, "-o", tmp, *objs, "-lcudart", "-lpthread"],
                   check=True)
    os.replace(tmp, so)
    return so


BOUNDS_SO = os.path.join(LIBDIR, "bounds", "liblbm_gb300.so")


def build_bounds_check(force: bool = False) -> str:
    """The bounds-check build: every computed population, index-record,
    row-word and row-start offset range-checked before the access (the
    device flag's bit 1 on a miss, lbm_device_flags).  A debugging aid, not
    loaded by the package."""
    return build_lbm(force, ["-DLBM_BOUNDS_CHECK"], out=BOUNDS_SO)


def build_all(force: bool = False) -> None:
    build_geometry(force)
    build_lbm(force)
