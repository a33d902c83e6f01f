"""ctypes binding of liblbm_gb300.so (the C ABI in include/lbm.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  There is no CPU fallback; if the library cannot be loaded or no
CUDA device is present the calls raise.

    solver = LBMSolver(mask, set_="B", tau=1.0, force=(1e-6, 0, 0))
    solver.run_to_convergence(1e-9)
    k = solver.permeability()          # eq. (perm_calc), lattice units
"""
from __future__ import annotations

import ctypes as C
import json
import math
import os
import time

import numpy as np

from . import _build

SET_A, SET_B, SET_C, SET_D, SET_E, SET_SRT = range(6)
SET_NAMES = {"A": SET_A, "B": SET_B, "C": SET_C, "D": SET_D, "E": SET_E, "SRT": SET_SRT}
FP64, FP32, FP16 = 0, 1, 2
PRECISIONS = {"fp64": FP64, "fp32": FP32, "fp16": FP16}
AB, AA, SPARSE = 0, 1, 2
LAYOUTS = {"ab": AB, "aa": AA, "sparse": SPARSE}

ERRORS = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ENOTCONV",
          -5: "EUNSTABLE", -6: "ETIMEOUT", -7: "ENOSTATE", -8: "EIO"}


class LBMError(RuntimeError):
    def __init__(self, code: int, what: str):
        msg = f"{what}: {ERRORS.get(code, code)} ({lib().lbm_strerror(code).decode()})"
        if code == -3:
            msg += f" [{lib().lbm_last_cuda_error().decode()}]"
        super().__init__(msg)
        self.code = code


class Grad(C.Structure):
    _fields_ = [("dk_dtau", C.c_double), ("dk_dLambda", C.c_double),
                ("dk_dLambda_q", C.c_double), ("dk_dLambda_m", C.c_double),
                ("dk_dF", C.c_double * 3), ("dk_ds", C.c_double * 6), ("k", C.c_double),
                ("iterations", C.c_int64), ("residual", C.c_double)]


class Check(C.Structure):
    _fields_ = [("step", C.c_int64), ("U", C.c_double), ("change", C.c_double)]


class LatticeDesc(C.Structure):
    _fields_ = [("mask", C.c_void_p), ("dims", C.c_int32 * 3), ("set", C.c_int32),
                ("tau", C.c_double), ("Lambda", C.c_double), ("s", C.c_double * 19),
                ("force", C.c_double * 3)]


class BatchOptions(C.Structure):
    _fields_ = [("precision", C.c_int32), ("layout", C.c_int32), ("nodes_per_thread", C.c_int32),
                ("check_interval", C.c_int32), ("linear_eq", C.c_int32), ("max_steps", C.c_int64),
                ("cuda_stream", C.c_void_p), ("use_graph", C.c_int32),
                ("barrier_timeout_ms", C.c_int32), ("test_skip_block", C.c_int32),
                ("stop_rule", C.c_int32), ("solo", C.c_int32), ("schedule", C.c_int32)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("layout", C.c_int32), ("check_interval", C.c_int32),
                ("linear_eq", C.c_int32), ("max_steps", C.c_int64), ("cuda_stream", C.c_void_p),
                ("fp16_scale_log2", C.c_int32), ("block_size", C.c_int32),
                ("stop_rule", C.c_int32), ("bounceback", C.c_int32),
                ("pressure_x", C.c_int32), ("symmetry", C.c_int32),
                ("rho_in", C.c_double), ("rho_out", C.c_double), ("collision", C.c_int32),
                ("index_width", C.c_int32)]


_lib = None


def lib():
    """Loads liblbm_gb300.so, building it in-tree if it is missing."""
    global _lib
    if _lib is None:
        path = _build.LBM_SO
        if not os.path.exists(path):
            _build.build_lbm()
        L = C.CDLL(path)
        vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
        dp = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
        u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
        sig = {
            "lbm_default_options": (None, [C.POINTER(Options)]),
            "lbm_rates": (C.c_int, [i32, dbl, dbl, dp]),
            "lbm_create": (C.c_int, [C.POINTER(vp), u8p, i32p, i32, dbl, dbl, dp,
                                     C.POINTER(Options)]),
            "lbm_create_rates": (C.c_int, [C.POINTER(vp), u8p, i32p, dp, dp, C.POINTER(Options)]),
            "lbm_destroy": (None, [vp]),
            "lbm_step": (C.c_int, [vp, i64]),
            "lbm_run_to_convergence": (C.c_int, [vp, dbl, C.POINTER(i64)]),
            "lbm_mean_velocity": (C.c_int, [vp, dp]),
            "lbm_permeability": (C.c_int, [vp, dp]),
            "lbm_velocity": (C.c_int, [vp, vp]),
            "lbm_get_populations": (C.c_int, [vp, vp]),
            "lbm_set_populations": (C.c_int, [vp, vp]),
            "lbm_get_populations_at": (C.c_int, [vp, vp, i64, vp]),
            "lbm_link_counts": (C.c_int, [vp, C.POINTER(i64), vp]),
            "lbm_sparse_tables": (C.c_int, [vp, vp, vp, vp]),
            "lbm_steps_done": (i64, [vp]),
            "lbm_kernel_launches": (i64, [vp]),
            "lbm_save": (C.c_int, [vp, C.c_char_p]),
            "lbm_load": (C.c_int, [C.POINTER(vp), C.c_char_p, C.POINTER(Options)]),
            "lbm_adjoint": (C.c_int, [vp, dbl, i64, C.POINTER(Grad)]),
            "lbm_adjoint_transient": (C.c_int, [vp, i64, C.POINTER(Grad)]),
            "lbm_mean_velocity_noalloc": (C.c_int, [vp, vp, i32p, dp, vp, vp]),
            "lbm_converged_velocity": (C.c_int, [vp, dp]),
            "lbm_device_flags": (C.c_int, [vp, C.POINTER(i32)]),
            "lbm_convergence_history": (C.c_int, [vp, C.POINTER(Check), i64,
                                                  C.POINTER(i64)]),
            "lbm_converged_permeability": (C.c_int, [vp, dp]),
            "lbm_batch_default_options": (None, [C.POINTER(BatchOptions)]),
            "lbm_batch_create": (C.c_int, [C.POINTER(vp), i32, C.POINTER(LatticeDesc),
                                           C.POINTER(BatchOptions)]),
            "lbm_batch_run": (C.c_int, [vp, dbl, vp, vp]),
            "lbm_batch_permeability": (C.c_int, [vp, vp]),
            "lbm_batch_mean_velocity": (C.c_int, [vp, vp]),
            "lbm_batch_config": (C.c_int, [vp, vp, vp]),
            "lbm_batch_lattice": (vp, [vp, i32]),
            "lbm_batch_kernel_launches": (i64, [vp]),
            "lbm_batch_schedule_counts": (C.c_int, [vp, C.POINTER(i64), C.POINTER(i64)]),
            "lbm_batch_destroy": (None, [vp]),
            "lbm_strerror": (C.c_char_p, [C.c_int]),
            "lbm_last_cuda_error": (C.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _json_float(v):
    v = float(v)
    return v if math.isfinite(v) else None


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise LBMError(rc, what)


def rates(set_: int | str, tau: float, Lambda: float = 3.0 / 16.0) -> np.ndarray:
    """Table 2 relaxation rates s[19] as the library computes them."""
    s = np.zeros(19)
    _check(lib().lbm_rates(SET_NAMES[set_] if isinstance(set_, str) else int(set_), float(tau),
                           float(Lambda), s), "lbm_rates")
    return s


def default_options() -> Options:
    o = Options()
    lib().lbm_default_options(C.byref(o))
    return o


class LBMSolver:
    """One lattice on the current CUDA device (one context = one C-ABI handle).

    mask: uint8 [Lz, Ly, Lx], 1 = solid.  Either (set_, tau, Lambda) or
    explicit rates s[19].  stream: a cudaStream_t handle (int) or a
    torch.cuda.Stream; None lets the library create its own stream.
    bounceback: "halfway" (default) or "fullway" (the paper's scheme; AB
    layout only).  pressure: (rho_in, rho_out) makes the x faces Zou-He
    density boundaries (force must be 0); symmetry: "y", "z" or "yz" makes
    those faces mirror planes (AB layout, halfway bounceback).  collision:
    "auto" (link-basis TRT where the rates allow, MRT otherwise) or "mrt".
    index_width: 0 (automatic) or 64 (64-bit population offsets even where
    32 bits would do; the path of very large lattices, bitwise the same).
    """

    def __init__(self, mask, set_="B", tau=1.0, Lambda=3.0 / 16.0, force=(1e-6, 0.0, 0.0), *,
                 rates_=None, precision="fp32", layout="aa", check_interval=100,
                 linear_eq=False, max_steps=1_000_000, stream=None, fp16_scale_log2=0,
                 block_size=0, stop_rule=0, bounceback="halfway", pressure=None, symmetry="",
                 collision="auto", index_width=0):
        self.mask = np.ascontiguousarray(mask, np.uint8)
        if self.mask.ndim != 3:
            raise ValueError("mask must be [Lz, Ly, Lx]")
        self.dims = np.array(self.mask.shape[::-1], np.int32)
        self.N = int(self.mask.size)
        self.force = np.ascontiguousarray(force, np.float64)
        o = default_options()
        o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        o.layout = LAYOUTS[layout] if isinstance(layout, str) else int(layout)
        o.check_interval = int(check_interval)
        o.linear_eq = int(bool(linear_eq))
        o.max_steps = int(max_steps)
        o.fp16_scale_log2 = int(fp16_scale_log2)
        o.block_size = int(block_size)
        o.stop_rule = int(stop_rule)
        o.bounceback = {"halfway": 0, "fullway": 1}[bounceback] if isinstance(bounceback, str) \
            else int(bounceback)
        if pressure is not None:
            o.pressure_x = 1
            o.rho_in, o.rho_out = (float(v) for v in pressure)
        o.symmetry = (1 if "y" in symmetry else 0) | (2 if "z" in symmetry else 0)
        o.collision = {"auto": 0, "mrt": 1}[collision]
        o.index_width = int(index_width)
        if stream is not None:
            o.cuda_stream = int(getattr(stream, "cuda_stream", stream))
        self.options = o
        h = C.c_void_p()
        if rates_ is not None:
            s = np.ascontiguousarray(rates_, np.float64)
            rc = lib().lbm_create_rates(C.byref(h), self.mask, self.dims, s, self.force, C.byref(o))
            self.tau = 1.0 / s[9]
        else:
            st = SET_NAMES[set_] if isinstance(set_, str) else int(set_)
            rc = lib().lbm_create(C.byref(h), self.mask, self.dims, st, float(tau), float(Lambda),
                                  self.force, C.byref(o))
            self.tau = float(tau)
        _check(rc, "lbm_create")
        self._h = h

    @classmethod
    def load(cls, path: str, stream=None) -> "LBMSolver":
        h = C.c_void_p()
        o = default_options()
        if stream is not None:
            o.cuda_stream = int(getattr(stream, "cuda_stream", stream))
        _check(lib().lbm_load(C.byref(h), path.encode(), C.byref(o)), "lbm_load")
        self = cls.__new__(cls)
        self._h = h
        with open(path, "rb") as fh:  # header: magic, version, dims, s[19], F[3]
            head = fh.read(8 + 4 + 12 + 152 + 24)
        dims = np.frombuffer(head[12:24], np.int32)
        s = np.frombuffer(head[24:176], np.float64)
        self.dims = dims.copy()
        self.N = int(np.prod(dims))
        self.force = np.frombuffer(head[176:200], np.float64).copy()
        self.tau = 1.0 / s[9]
        self.mask = None
        return self

    def close(self) -> None:
        if getattr(self, "_h", None):
            if getattr(self, "_owned", True):
                lib().lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------- stepping
    def step(self, n: int = 1) -> None:
        _check(lib().lbm_step(self._h, int(n)), "lbm_step")

    def run_to_convergence(self, tol: float, raise_on_failure: bool = True):
        """Returns (status code, steps taken by this call)."""
        steps = C.c_int64(0)
        t0 = time.perf_counter()
        rc = lib().lbm_run_to_convergence(self._h, float(tol), C.byref(steps))
        self._last_run = dict(status=ERRORS.get(rc, rc), tol=float(tol), steps=int(steps.value),
                              wall_s=time.perf_counter() - t0)
        if rc not in (0, -4) and raise_on_failure:
            raise LBMError(rc, "lbm_run_to_convergence")
        return rc, int(steps.value)

    def convergence_history(self) -> np.ndarray:
        """The checks of the last run_to_convergence (lbm_convergence_history):
        a structured array of (step, U along the drive, relative change)."""
        n = C.c_int64(0)
        _check(lib().lbm_convergence_history(self._h, None, 0, C.byref(n)),
               "lbm_convergence_history")
        buf = (Check * max(n.value, 1))()
        _check(lib().lbm_convergence_history(self._h, buf, n.value, C.byref(n)),
               "lbm_convergence_history")
        out = np.zeros(n.value, dtype=[("step", np.int64), ("U", np.float64),
                                       ("change", np.float64)])
        for i in range(n.value):
            out[i] = (buf[i].step, buf[i].U, buf[i].change)
        return out

    def run_record(self) -> dict:
        """A JSON-serialisable record of the last run_to_convergence: the
        configuration, the status, steps and wall time, every check of the
        stopping rule and the converged velocity and permeability."""
        o = self.options if hasattr(self, "options") else None
        last = getattr(self, "_last_run", None)
        rec = {
            "dims": [int(v) for v in self.dims],
            "tau": float(self.tau),
            "force": [float(v) for v in self.force],
            "precision": {v: k for k, v in PRECISIONS.items()}.get(o.precision) if o else None,
            "layout": {v: k for k, v in LAYOUTS.items()}.get(o.layout) if o else None,
            "stop_rule": int(o.stop_rule) if o else None,
            "check_interval": int(o.check_interval) if o else None,
            "run": last,
            "steps_total": self.steps,
            "kernel_launches": self.kernel_launches,
        }
        h = self.convergence_history()
        rec["history"] = [{"step": int(r["step"]), "U": _json_float(r["U"]),
                           "change": _json_float(r["change"])} for r in h]
        if last is not None and last["status"] in ("OK", "ENOTCONV") and len(h):
            rec["U_conv"] = [float(v) for v in self.converged_velocity()]
            rec["k_conv"] = [float(v) for v in self.converged_permeability()]
        return rec

    def write_run_record(self, path: str) -> None:
        with open(path, "w") as fh:
            json.dump(self.run_record(), fh, indent=1)
            fh.write("\n")

    # -------------------------------------------------------------- outputs
    def mean_velocity(self) -> np.ndarray:
        U = np.zeros(3)
        _check(lib().lbm_mean_velocity(self._h, U), "lbm_mean_velocity")
        return U

    def permeability(self) -> np.ndarray:
        k = np.zeros(3)
        _check(lib().lbm_permeability(self._h, k), "lbm_permeability")
        return k

    def device_flags(self) -> int:
        """Reads and clears the device flags (lbm_device_flags): 1 = a
        non-finite value was measured, 2 = an index out of range was skipped
        (bounds-check build only)."""
        f = C.c_int32(0)
        _check(lib().lbm_device_flags(self._h, C.byref(f)), "lbm_device_flags")
        return int(f.value)

    def converged_velocity(self) -> np.ndarray:
        """The mean velocity the last stopping-rule run stopped on."""
        U = np.zeros(3)
        _check(lib().lbm_converged_velocity(self._h, U), "lbm_converged_velocity")
        return U

    def converged_permeability(self) -> np.ndarray:
        k = np.zeros(3)
        _check(lib().lbm_converged_permeability(self._h, k), "lbm_converged_permeability")
        return k

    def velocity(self) -> np.ndarray:
        u = np.zeros(3 * self.N)
        _check(lib().lbm_velocity(self._h, u.ctypes.data), "lbm_velocity")
        return u.reshape((3,) + tuple(self.dims[::-1]))

    def get_populations(self) -> np.ndarray:
        f = np.zeros(19 * self.N)
        _check(lib().lbm_get_populations(self._h, f.ctypes.data), "lbm_get_populations")
        return f.reshape((19,) + tuple(self.dims[::-1]))

    def set_populations(self, f: np.ndarray) -> None:
        f = np.ascontiguousarray(f, np.float64).reshape(-1)
        if f.size != 19 * self.N:
            raise ValueError("populations must have 19*N entries")
        _check(lib().lbm_set_populations(self._h, f.ctypes.data), "lbm_set_populations")

    def get_populations_at(self, nodes) -> np.ndarray:
        """Post-collision populations f[len(nodes), 19] at node indices."""
        nodes = np.ascontiguousarray(nodes, np.int64).reshape(-1)
        f = np.zeros((len(nodes), 19))
        _check(lib().lbm_get_populations_at(self._h, nodes.ctypes.data, len(nodes), f.ctypes.data),
               "lbm_get_populations_at")
        return f

    def link_counts(self):
        nf = C.c_int64(0)
        links = np.zeros(19, np.int64)
        _check(lib().lbm_link_counts(self._h, C.byref(nf), links.ctypes.data), "lbm_link_counts")
        return int(nf.value), links

    def sparse_tables(self):
        nf, _ = self.link_counts()
        fi = np.zeros(max(nf, 1), np.int32)
        nbr = np.zeros(max(18 * nf, 1), np.int32)
        bb = np.zeros(max(nf, 1), np.uint32)
        _check(lib().lbm_sparse_tables(self._h, fi.ctypes.data, nbr.ctypes.data, bb.ctypes.data),
               "lbm_sparse_tables")
        return fi[:nf], nbr[: 18 * nf].reshape(18, nf), bb[:nf]

    @property
    def steps(self) -> int:
        return int(lib().lbm_steps_done(self._h))

    @property
    def kernel_launches(self) -> int:
        return int(lib().lbm_kernel_launches(self._h))

    def save(self, path: str) -> None:
        _check(lib().lbm_save(self._h, path.encode()), "lbm_save")

    def adjoint(self, tol: float = 1e-8, max_iter: int = 1_000_000) -> dict:
        """Gradient of the converged permeability along the drive (lbm_adjoint)."""
        g = Grad()
        _check(lib().lbm_adjoint(self._h, float(tol), int(max_iter), C.byref(g)), "lbm_adjoint")
        return _grad_dict(g)

    def adjoint_transient(self, n: int) -> dict:
        """Gradient of the permeability after n more steps
        (lbm_adjoint_transient); the solver advances n steps."""
        g = Grad()
        _check(lib().lbm_adjoint_transient(self._h, int(n), C.byref(g)), "lbm_adjoint_transient")
        return _grad_dict(g)


def _grad_dict(g) -> dict:
    return {"dtau": g.dk_dtau, "dLambda": g.dk_dLambda, "dLambda_q": g.dk_dLambda_q,
            "dLambda_m": g.dk_dLambda_m, "dF": np.array(list(g.dk_dF)),
            "ds": np.array(list(g.dk_ds)), "k": g.k, "iterations": int(g.iterations),
            "residual": g.residual}


class LBMBatch:
    """Many lattices stepped together by the batched persistent kernel
    (lbm_batch_*).  `lattices` is a list of dicts with keys mask, and either
    set_/tau/Lambda or rates_, and force.  layout None lets the autotuner pick
    dense AA or sparse per distinct image; nodes_per_thread 0 likewise, and
    then a lattice may run alone with the single-lattice kernels where that is
    faster (solo "auto"; "never", or "always" for every autotuned lattice).
    schedule: "auto" (lattices of at least 10^5 units on their own
    graph-replayed kernels, the rest in one persistent launch),
    "persistent", or "stepwise" (grouped multi-lattice launches per step)."""

    def __init__(self, lattices, precision="fp32", layout=None, nodes_per_thread=0,
                 check_interval=100, linear_eq=False, max_steps=1_000_000, stream=None,
                 use_graph=True, barrier_timeout_ms=2000, test_skip_block=-1, stop_rule=0,
                 solo="auto", schedule="auto"):
        self.masks = [np.ascontiguousarray(l["mask"], np.uint8) for l in lattices]
        n = len(lattices)
        descs = (LatticeDesc * n)()
        for i, (l, m) in enumerate(zip(lattices, self.masks)):
            d = descs[i]
            d.mask = m.ctypes.data
            for a, v in enumerate(m.shape[::-1]):
                d.dims[a] = v
            if l.get("rates_") is not None:
                d.set = -1
                for k, v in enumerate(np.asarray(l["rates_"], np.float64)):
                    d.s[k] = v
            else:
                st = l.get("set_", "B")
                d.set = SET_NAMES[st] if isinstance(st, str) else int(st)
                d.tau = float(l.get("tau", 1.0))
                d.Lambda = float(l.get("Lambda", 3.0 / 16.0))
            for a, v in enumerate(l.get("force", (1e-6, 0.0, 0.0))):
                d.force[a] = float(v)
        o = BatchOptions()
        lib().lbm_batch_default_options(C.byref(o))
        o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        o.layout = -1 if layout is None else (LAYOUTS[layout] if isinstance(layout, str) else int(layout))
        o.nodes_per_thread = int(nodes_per_thread)
        o.check_interval = int(check_interval)
        o.linear_eq = int(bool(linear_eq))
        o.max_steps = int(max_steps)
        o.use_graph = int(bool(use_graph))
        o.barrier_timeout_ms = int(barrier_timeout_ms)
        o.test_skip_block = int(test_skip_block)
        o.stop_rule = int(stop_rule)
        o.solo = {"never": 0, "auto": 1, "always": 2}[solo]
        o.schedule = {"auto": 0, "persistent": 1, "stepwise": 2}[schedule]
        if stream is not None:
            o.cuda_stream = int(getattr(stream, "cuda_stream", stream))
        h = C.c_void_p()
        _check(lib().lbm_batch_create(C.byref(h), n, descs, C.byref(o)), "lbm_batch_create")
        self._h = h
        self.n = n

    def close(self):
        if getattr(self, "_h", None):
            lib().lbm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, tol: float, raise_on_failure: bool = True):
        """Returns (steps[n], status[n])."""
        steps = np.zeros(self.n, np.int64)
        status = np.zeros(self.n, np.int32)
        rc = lib().lbm_batch_run(self._h, float(tol), steps.ctypes.data, status.ctypes.data)
        if rc != 0 and raise_on_failure:
            raise LBMError(rc, "lbm_batch_run")
        return (steps, status) if rc == 0 else rc

    def permeability(self) -> np.ndarray:
        k = np.zeros((self.n, 3))
        _check(lib().lbm_batch_permeability(self._h, k.ctypes.data), "lbm_batch_permeability")
        return k

    def mean_velocity(self) -> np.ndarray:
        U = np.zeros((self.n, 3))
        _check(lib().lbm_batch_mean_velocity(self._h, U.ctypes.data), "lbm_batch_mean_velocity")
        return U

    def config(self):
        lay = np.zeros(self.n, np.int32)
        npt = np.zeros(self.n, np.int32)
        _check(lib().lbm_batch_config(self._h, lay.ctypes.data, npt.ctypes.data), "lbm_batch_config")
        return lay, npt

    @property
    def kernel_launches(self) -> int:
        return int(lib().lbm_batch_kernel_launches(self._h))

    def schedule_counts(self):
        """(stepwise chunks, persistent chunks) run so far."""
        a, b = C.c_int64(0), C.c_int64(0)
        _check(lib().lbm_batch_schedule_counts(self._h, C.byref(a), C.byref(b)),
               "lbm_batch_schedule_counts")
        return int(a.value), int(b.value)

    def lattice(self, i: int) -> "LBMSolver":
        """Non-owning view of lattice i as a single-lattice solver."""
        h = lib().lbm_batch_lattice(self._h, int(i))
        if not h:
            raise IndexError(i)
        view = LBMSolver.__new__(LBMSolver)
        view._h = C.c_void_p(h)
        view._owned = False  # the batch owns the context
        view.mask = self.masks[i]
        view.dims = np.array(self.masks[i].shape[::-1], np.int32)
        view.N = int(self.masks[i].size)
        view._batch = self
        return view
