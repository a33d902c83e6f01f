"""Seeded synthetic voxel images (input generators shared by the tests, the
benchmark and the CUDA path; no lattice Boltzmann arithmetic here).

Masks are uint8 numpy arrays shaped [Lz, Ly, Lx] (x fastest), 1 = solid.
Geometries: simple-cubic / BCC / FCC sphere arrays (Sec. 3.1 names BCC and FCC
packings as periodic media), Boolean overlapping-sphere media standing in for
the random sphere pack of Sec. 4.3, a plane slit, a rectangular duct, and the
circular and triangular bores of Secs. 4.1-4.2.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _build

_lib = None

SC, BCC, FCC = 0, 1, 2
_KINDS = {"sc": SC, "bcc": BCC, "fcc": FCC}
_PER_CELL = {SC: 1, BCC: 2, FCC: 4}


def _L():
    global _lib
    if _lib is None:
        _build.build_geometry()
        L = C.CDLL(_build.GEOM_SO)
        u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
        L.geom_sphere_array.argtypes = [u8p, C.c_int, C.c_int, C.c_double]
        L.geom_radius_for_fraction.argtypes = [C.c_int, C.c_int, C.c_double]
        L.geom_radius_for_fraction.restype = C.c_double
        L.geom_boolean.argtypes = [u8p, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                   C.c_uint64, C.c_int64, C.POINTER(C.c_int64),
                                   C.POINTER(C.c_int64)]
        L.geom_slit.argtypes = [u8p, C.c_int, C.c_int, C.c_int, C.c_int]
        L.geom_duct.argtypes = [u8p, C.c_int, C.c_int, C.c_int]
        L.geom_pipe.argtypes = [u8p, C.c_int, C.c_int, C.c_int, C.c_double]
        L.geom_triangle.argtypes = [u8p, C.c_int, C.c_int, C.c_int, C.c_double]
        L.geom_fill_isolated.argtypes = [u8p, C.c_int, C.c_int, C.c_int]
        L.geom_fill_isolated.restype = C.c_int64
        L.geom_splitmix64.argtypes = [C.POINTER(C.c_uint64)]
        L.geom_splitmix64.restype = C.c_uint64
        for fn in ("geom_sphere_array", "geom_boolean", "geom_slit", "geom_duct",
                   "geom_pipe", "geom_triangle"):
            getattr(L, fn).restype = C.c_int
        _lib = L
    return _lib


def _check(rc: int) -> None:
    if rc != 0:
        raise ValueError("invalid geometry parameters")


def splitmix64(seed: int, n: int) -> np.ndarray:
    st = C.c_uint64(seed)
    return np.array([_L().geom_splitmix64(C.byref(st)) for _ in range(n)], dtype=np.uint64)


def radius_for_fraction(L: int, kind: str | int, c: float) -> float:
    k = _KINDS[kind] if isinstance(kind, str) else kind
    return float(_L().geom_radius_for_fraction(L, _PER_CELL[k], c))


def sphere_array(L: int, kind: str | int = "sc", r: float | None = None,
                 c: float | None = None) -> np.ndarray:
    """Periodic cubic cell of edge L; give either the radius r or the solid
    fraction c (before overlap) of the sphere array."""
    k = _KINDS[kind] if isinstance(kind, str) else kind
    if r is None:
        r = radius_for_fraction(L, k, c)
    m = np.zeros((L, L, L), np.uint8)
    _check(_L().geom_sphere_array(m, L, k, float(r)))
    return m


def boolean(dims, r: float, porosity: float, seed: int, max_spheres: int = 0,
            connected: bool = False):
    """Overlapping monodisperse spheres at SplitMix64(seed) centres until the
    porosity is <= target.  connected=True then fills enclosed pores (see
    fill_isolated).  Returns (mask, n_spheres)."""
    Lx, Ly, Lz = (dims, dims, dims) if np.isscalar(dims) else dims
    m = np.zeros((Lz, Ly, Lx), np.uint8)
    ns, nsol = C.c_int64(0), C.c_int64(0)
    _check(_L().geom_boolean(m, Lx, Ly, Lz, float(r), float(porosity), C.c_uint64(seed),
                             int(max_spheres), C.byref(ns), C.byref(nsol)))
    if connected:
        fill_isolated(m)
    return m, int(ns.value)


def fill_isolated(mask: np.ndarray) -> int:
    """In place: fills as solid every fluid cluster except the largest, with
    clusters joined by D3Q19 links under periodic wrap (the usual removal of
    enclosed pores from a segmented image).  Returns the voxels filled."""
    if not (mask.flags.c_contiguous and mask.dtype == np.uint8):
        raise ValueError("mask must be a C-contiguous uint8 array")
    Lz, Ly, Lx = mask.shape
    n = int(_L().geom_fill_isolated(mask, Lx, Ly, Lz))
    if n < 0:
        raise ValueError("fill_isolated failed")
    return n


def slit(H: int, W: int = 1, Lx: int = 1, Lz: int = 1) -> np.ndarray:
    m = np.zeros((Lz, H + W, Lx), np.uint8)
    _check(_L().geom_slit(m, Lx, H, W, Lz))
    return m


def duct(a: int, b: int | None = None, Lx: int = 1) -> np.ndarray:
    b = a if b is None else b
    m = np.zeros((b + 1, a + 1, Lx), np.uint8)
    _check(_L().geom_duct(m, Lx, a, b))
    return m


def pipe(D: float, Ly: int, Lz: int | None = None, Lx: int = 1) -> np.ndarray:
    Lz = Ly if Lz is None else Lz
    m = np.zeros((Lz, Ly, Lx), np.uint8)
    _check(_L().geom_pipe(m, Lx, Ly, Lz, float(D)))
    return m


def triangle(l: float, Ly: int, Lz: int | None = None, Lx: int = 1) -> np.ndarray:
    Lz = Ly if Lz is None else Lz
    m = np.zeros((Lz, Ly, Lx), np.uint8)
    _check(_L().geom_triangle(m, Lx, Ly, Lz, float(l)))
    return m


def pad_x(mask: np.ndarray, layers: int = 5) -> np.ndarray:
    """Fluid layers before and after a sample along x, the flow direction
    (Sec. 2.4: inlet and outlet padded with 5 fluid-only layers)."""
    Lz, Ly, _ = mask.shape
    pad = np.zeros((Lz, Ly, layers), np.uint8)
    return np.ascontiguousarray(np.concatenate([pad, np.asarray(mask, np.uint8), pad], axis=2))


def random_mask(dims, solid_fraction: float, seed: int) -> np.ndarray:
    """Independent random voxels (structure tests on tiny lattices)."""
    Lx, Ly, Lz = (dims, dims, dims) if np.isscalar(dims) else dims
    rng = np.random.default_rng(seed)
    return (rng.random((Lz, Ly, Lx)) < solid_fraction).astype(np.uint8)
