"""FP64 CPU oracle for the D3Q19-MRT permeability solver (Rao & Schaefer,
arXiv:1902.11193).

TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the benchmark's
CPU-baseline arm load it; the product package never imports it.  It shares no
code with the CUDA path: the C source ``oracle.c`` is the whole method, this
module only marshals numpy arrays into it.

Functions follow the paper's equations:
  rates            Table 2 (Sets A-E, SRT), eq. (MRT params), eq. (Magic param)
  meq              eq. (MRT Equi), read so that m^eq = M f^eq
  guo_populations  eq. (Guo_Forcing)
  force_moments    m^F = M . F_i (Sec. 2.2.1)
  collide          eq. (MRT-LBE) for one node
  links            fluid list, pull neighbours, bounceback bits (halfway BB)
  Solver           pull stream + collide; mean velocity; eq. (perm_calc);
                   stopping rule eq. (convergence)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")

SET_A, SET_B, SET_C, SET_D, SET_E, SET_SRT = range(6)
SET_NAMES = {"A": SET_A, "B": SET_B, "C": SET_C, "D": SET_D, "E": SET_E, "SRT": SET_SRT}


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (OpenMP over z-planes)."""
    src = os.path.join(_HERE, "oracle.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= max(
        os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "oracle.h"))
    ):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.run(
        ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-D_DEFAULT_SOURCE",
         "-o", tmp, src, "-lm"],
        check=True,
    )
    os.replace(tmp, _SO)
    return _SO


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_SO)
        dp = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
        u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
        L.ora_lattice.argtypes = [i32p, dp, i32p]
        L.ora_moment_matrix.argtypes = [dp]
        L.ora_rates.argtypes = [C.c_int, C.c_double, C.c_double, dp]
        L.ora_rates.restype = C.c_int
        L.ora_meq.argtypes = [C.c_double, dp, C.c_int, dp]
        L.ora_guo_populations.argtypes = [dp, dp, C.c_int, dp]
        L.ora_force_moments.argtypes = [dp, dp, C.c_int, dp]
        L.ora_collide.argtypes = [dp, dp, dp, C.c_int, dp]
        L.ora_links.argtypes = [u8p, i32p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.ora_links.restype = C.c_int64
        L.ora_trt_collide.argtypes = [dp, C.c_double, C.c_double, dp, C.c_int, dp]
        L.ora_trt_collide.restype = None
        L.ora_flags.argtypes = [u8p, i32p, u8p]
        L.ora_flags.restype = C.c_int64
        L.ora_set_bounceback.argtypes = [C.c_void_p, C.c_int]
        L.ora_set_bounceback.restype = C.c_int
        L.ora_set_domain.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_int]
        L.ora_set_domain.restype = C.c_int
        L.ora_create.argtypes = [u8p, i32p, dp, dp, C.c_int]
        L.ora_create.restype = C.c_void_p
        L.ora_destroy.argtypes = [C.c_void_p]
        L.ora_step.argtypes = [C.c_void_p, C.c_int64, C.c_void_p]
        L.ora_mean_velocity.argtypes = [C.c_void_p, dp]
        L.ora_velocity.argtypes = [C.c_void_p, dp]
        L.ora_get_f.argtypes = [C.c_void_p, dp]
        L.ora_set_f.argtypes = [C.c_void_p, dp]
        L.ora_steps_done.argtypes = [C.c_void_p]
        L.ora_steps_done.restype = C.c_int64
        L.ora_run_to_convergence.argtypes = [C.c_void_p, C.c_double, C.c_int64, C.c_int64,
                                             C.POINTER(C.c_int64), dp]
        L.ora_run_to_convergence.restype = C.c_int
        L.ora_set_threads.argtypes = [C.c_int]
        L.ora_get_threads.restype = C.c_int
        L.ora_run_to_convergence_rule.argtypes = [C.c_void_p, C.c_double, C.c_int64, C.c_int64,
                                                  C.c_int, C.POINTER(C.c_int64), dp]
        L.ora_run_to_convergence_rule.restype = C.c_int
        L.ora_rates_magic.argtypes = [C.c_double, C.c_double, C.c_double, dp]
        L.ora_rates_magic.restype = C.c_int
        L.ora_stream_field.argtypes = [C.c_void_p, dp, dp]
        L.ora_unstream_field.argtypes = [C.c_void_p, dp, dp]
        L.ora_adjoint_apply.argtypes = [C.c_void_p, dp, dp]
        L.ora_adjoint.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_double,
                                  C.c_int64, C.c_int64, dp, C.POINTER(C.c_int64)]
        L.ora_adjoint.restype = C.c_int
        L.ora_adjoint_transient.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double,
                                            C.c_int64, dp]
        L.ora_adjoint_transient.restype = C.c_int
        _lib = L
    return _lib


def set_threads(n: int) -> None:
    lib().ora_set_threads(int(n))


def get_threads() -> int:
    return int(lib().ora_get_threads())


def lattice():
    """(c[19,3] int, w[19], opp[19]) of the D3Q19 set in the oracle's order."""
    c = np.zeros(57, np.int32)
    w = np.zeros(19)
    opp = np.zeros(19, np.int32)
    lib().ora_lattice(c, w, opp)
    return c.reshape(19, 3), w, opp


def moment_matrix() -> np.ndarray:
    M = np.zeros(361)
    lib().ora_moment_matrix(M)
    return M.reshape(19, 19)


def rates(set_: int | str, tau: float, Lambda: float = 3.0 / 16.0) -> np.ndarray:
    if isinstance(set_, str):
        set_ = SET_NAMES[set_]
    s = np.zeros(19)
    if lib().ora_rates(int(set_), float(tau), float(Lambda), s) != 0:
        raise ValueError(f"invalid rate parameters set={set_} tau={tau} Lambda={Lambda}")
    return s


def rates_magic(tau: float, Lq: float, Lm: float) -> np.ndarray:
    """Sets B/D/E with the odd rates given by their magic parameters."""
    s = np.zeros(19)
    if lib().ora_rates_magic(float(tau), float(Lq), float(Lm), s) != 0:
        raise ValueError("invalid magic parameters")
    return s


GRAD_KEYS = ("dtau", "dLambda", "dLambda_q", "dLambda_m", "dFx", "dFy", "dFz")


def meq(rho: float, j, linear: bool = False) -> np.ndarray:
    out = np.zeros(19)
    lib().ora_meq(float(rho), np.ascontiguousarray(j, np.float64), int(linear), out)
    return out


def guo_populations(u, F, linear: bool = False) -> np.ndarray:
    out = np.zeros(19)
    lib().ora_guo_populations(np.ascontiguousarray(u, np.float64),
                              np.ascontiguousarray(F, np.float64), int(linear), out)
    return out


def force_moments(u, F, linear: bool = False) -> np.ndarray:
    out = np.zeros(19)
    lib().ora_force_moments(np.ascontiguousarray(u, np.float64),
                            np.ascontiguousarray(F, np.float64), int(linear), out)
    return out


def collide(f, s, F, linear: bool = False) -> np.ndarray:
    out = np.zeros(19)
    lib().ora_collide(np.ascontiguousarray(f, np.float64), np.ascontiguousarray(s, np.float64),
                      np.ascontiguousarray(F, np.float64), int(linear), out)
    return out


def trt_collide(f, s_plus, s_minus, F, linear: bool = False) -> np.ndarray:
    out = np.zeros(19)
    lib().ora_trt_collide(np.ascontiguousarray(f, np.float64), float(s_plus), float(s_minus),
                          np.ascontiguousarray(F, np.float64), int(linear), out)
    return out


def links(mask: np.ndarray):
    """Returns (fluid_idx[Nf], nbr[18, Nf], bbmask[Nf] uint32, links[19] int64)."""
    mask = np.ascontiguousarray(mask, np.uint8)
    dims = np.array(mask.shape[::-1], np.int32)
    Nf = int((mask == 0).sum())
    fi = np.zeros(max(Nf, 1), np.int32)
    nbr = np.zeros(max(18 * Nf, 1), np.int32)
    bb = np.zeros(max(Nf, 1), np.uint32)
    lk = np.zeros(19, np.int64)
    n = lib().ora_links(mask, dims, fi.ctypes.data, nbr.ctypes.data, bb.ctypes.data,
                        lk.ctypes.data)
    assert n == Nf
    return fi[:Nf], nbr[: 18 * Nf].reshape(18, Nf), bb[:Nf], lk


def flags(mask: np.ndarray) -> np.ndarray:
    """Voxel flags of the image analysis: 0 fluid, 1 bounceback voxel (solid
    with a fluid link neighbour), 2 other solid; shape of the mask."""
    mask = np.ascontiguousarray(mask, np.uint8)
    dims = np.array(mask.shape[::-1], np.int32)
    out = np.zeros_like(mask)
    lib().ora_flags(mask, dims, out)
    return out


class Solver:
    """Plain FP64 solver on a mask [Lz, Ly, Lx] (1 = solid).  bounceback
    "halfway" (default) or "fullway" (the paper's scheme of Sec. 3)."""

    def __init__(self, mask: np.ndarray, s, F, linear: bool = False, bounceback: str = "halfway"):
        self.mask = np.ascontiguousarray(mask, np.uint8)
        self.dims = np.array(self.mask.shape[::-1], np.int32)
        self.N = int(self.mask.size)
        self.F = np.ascontiguousarray(F, np.float64)
        self.s = np.ascontiguousarray(s, np.float64)
        self._h = lib().ora_create(self.mask, self.dims, self.s, self.F, int(linear))
        if not self._h:
            raise ValueError("oracle create failed")
        mode = {"halfway": 0, "fullway": 1}[bounceback]
        if lib().ora_set_bounceback(self._h, mode) != 0:
            raise ValueError("bad bounceback mode")

    def set_domain(self, pressure_x=False, rho_in=1.0, rho_out=1.0, symmetry_y=False,
                   symmetry_z=False):
        """Bounded domain: Zou-He density faces in x, symmetry planes in y and/or z."""
        sym = (1 if symmetry_y else 0) | (2 if symmetry_z else 0)
        if lib().ora_set_domain(self._h, int(bool(pressure_x)), float(rho_in), float(rho_out),
                                sym) != 0:
            raise ValueError("invalid domain settings")

    def close(self):
        if self._h:
            lib().ora_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1, want_U: bool = False):
        U = np.zeros(3)
        lib().ora_step(self._h, int(n), U.ctypes.data if want_U else None)
        return U if want_U else None

    def mean_velocity(self) -> np.ndarray:
        U = np.zeros(3)
        lib().ora_mean_velocity(self._h, U)
        return U

    def velocity(self) -> np.ndarray:
        u = np.zeros(3 * self.N)
        lib().ora_velocity(self._h, u)
        return u.reshape((3,) + self.mask.shape)

    def get_f(self) -> np.ndarray:
        f = np.zeros(19 * self.N)
        lib().ora_get_f(self._h, f)
        return f.reshape((19,) + self.mask.shape)

    def set_f(self, f: np.ndarray) -> None:
        lib().ora_set_f(self._h, np.ascontiguousarray(f, np.float64).reshape(-1))

    @property
    def steps(self) -> int:
        return int(lib().ora_steps_done(self._h))

    def run_to_convergence(self, tol: float, K: int = 1, max_steps: int = 10**6, rule: int = 0):
        """Stopping rule of eq. (convergence); rule 1 applies it to the mean
        over two consecutive steps.  Returns (rc, steps, U stopped on)."""
        steps = C.c_int64(0)
        U = np.zeros(3)
        rc = lib().ora_run_to_convergence_rule(self._h, float(tol), int(K), int(max_steps),
                                               int(rule), C.byref(steps), U)
        return rc, int(steps.value), U

    def stream_field(self, f: np.ndarray) -> np.ndarray:
        out = np.zeros(19 * self.N)
        lib().ora_stream_field(self._h, np.ascontiguousarray(f, np.float64).reshape(-1), out)
        return out.reshape((19,) + self.mask.shape)

    def unstream_field(self, f: np.ndarray) -> np.ndarray:
        out = np.zeros(19 * self.N)
        lib().ora_unstream_field(self._h, np.ascontiguousarray(f, np.float64).reshape(-1), out)
        return out.reshape((19,) + self.mask.shape)

    def adjoint_apply(self, psi: np.ndarray) -> np.ndarray:
        """J_C(h)^T S^T psi at the current state (h = S f*)."""
        out = np.zeros(19 * self.N)
        lib().ora_adjoint_apply(self._h, np.ascontiguousarray(psi, np.float64).reshape(-1), out)
        return out.reshape((19,) + self.mask.shape)

    def adjoint(self, set_, tau: float, Lambda: float = 3.0 / 16.0, tol: float = 1e-12,
                K: int = 10, max_iter: int = 10**6):
        """Steady fixed-point adjoint: returns (rc, gradient dict, iterations)."""
        st = SET_NAMES[set_] if isinstance(set_, str) else int(set_)
        g = np.zeros(7)
        it = C.c_int64(0)
        rc = lib().ora_adjoint(self._h, st, float(tau), float(Lambda), float(tol), int(K),
                               int(max_iter), g, C.byref(it))
        return rc, dict(zip(GRAD_KEYS, g)), int(it.value)

    def adjoint_transient(self, set_, tau: float, Lambda: float = 3.0 / 16.0, n: int = 100):
        """Gradient of k after n more steps (the solver advances n steps):
        returns (rc, gradient dict)."""
        st = SET_NAMES[set_] if isinstance(set_, str) else int(set_)
        g = np.zeros(7)
        rc = lib().ora_adjoint_transient(self._h, st, float(tau), float(Lambda), int(n), g)
        return rc, dict(zip(GRAD_KEYS, g))

    def permeability(self, tau: float) -> np.ndarray:
        """eq. (perm_calc) with body forcing: k_j = nu <u_j> / F_j, nu = (tau - 1/2)/3."""
        U = self.mean_velocity()
        nu = (tau - 0.5) / 3.0
        with np.errstate(divide="ignore", invalid="ignore"):
            return np.where(self.F != 0, nu * U / np.where(self.F != 0, self.F, 1.0), np.nan)
