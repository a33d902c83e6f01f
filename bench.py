"""Benchmark of the D3Q19-MRT permeability hot path on GB300.

Workload (default): the 512^3 Boolean overlapping-sphere medium (radius 10
voxels, SplitMix64 seed 1902_11193 + 1, porosity 0.40, periodic), Set B,
tau = 1, body force 1e-6 along x, FP32 shifted populations.  One "step" is
one time step of the production loop of lbm_run_to_convergence (fused
stream-collide on every step, the fused mean-velocity reduction and stopping
rule on the last two steps of every 100-step chunk).  Value = fluid-node
updates per second (fluid MLUPS), summed over ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--layout sparse|aa|ab]
  python bench.py --impl reference      # the FP64 CPU oracle, host cores

Multi-GPU: one process per GPU, independent replicas of the same lattice
(weak scaling); the lattice is not domain-decomposed, so ranks exchange
nothing but the timing barrier.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_PER_UPDATE = {"fp32": 152, "fp16": 76, "fp64": 304}  # 19 reads + 19 writes
SEED = 1902_11193 + 1


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=50)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--size", type=int, default=512)
    p.add_argument("--layout", default="sparse", choices=["sparse", "aa", "ab"])
    p.add_argument("--precision", default="fp32", choices=["fp32", "fp16", "fp64"])
    p.add_argument("--block-size", type=int, default=0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-extra", action="store_true",
                   help="skip the other-layout and permeability-error legs")
    p.add_argument("--sweep", default="subset", choices=["none", "subset", "full"],
                   help="batched parameter sweep vs the same lattices one by one")
    p.add_argument("--adjoint", action="store_true", default=True)
    p.add_argument("--no-adjoint", dest="adjoint", action="store_false")
    p.add_argument("--adjoint-size", type=int, default=128,
                   help="edge of the adjoint leg's Boolean medium (r = 6, porosity 0.35)")
    p.add_argument("--adjoint-sets", default="B,D,E3/16,E3/8",
                   help="rate sets of the adjoint grid (E with its magic parameter)")
    p.add_argument("--adjoint-taus", default="0.8,1.0,1.3", help="taus of the adjoint grid")
    p.add_argument("--no-transient", action="store_true",
                   help="skip the transient adjoint of the adjoint leg")
    p.add_argument("--large", action="store_true", default=True,
                   help="1024^3 low-porosity sparse leg, FP32 vs FP16 storage")
    p.add_argument("--no-large", dest="large", action="store_false")
    p.add_argument("--channels", default="lowres", choices=["none", "lowres", "full"],
                   help="the paper's channel study as one batch: lowres = circular bores "
                        "D = 32, 64 and the 64^2 resolution series; full adds D = 128 and the "
                        "triangular bore")
    return p.parse_args()


def workload(size):
    from paper_1902_11193_gb300 import geometry

    mask, nspheres = geometry.boolean(size, 10, 0.40, seed=SEED)
    return mask, nspheres


def workload_name(args):
    return (f"boolean-{args.size}^3 r=10 porosity=0.40 seed={SEED}; D3Q19-MRT Set B tau=1 "
            f"F=1e-6 x; {args.precision} shifted; {args.layout} layout")


KERNEL_SOURCES = ("lbm_kernels.cu", "lbm_step.cuh", "lbm_collide.cuh", "lbm_sparse.cuh",
                  "lbm_internal.cuh")


def kernel_source_hash():
    """Hash of the stream-collide sources with comments and blank lines
    removed, so that a change to a comment keeps the measured traffic."""
    import hashlib
    import re

    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1902_11193_gb300", "csrc", name)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        code = "\n".join(line.rstrip() for line in text.splitlines() if line.strip())
        h.update(code.encode())
    return h.hexdigest()[:16]


def measured_traffic(layout, precision, nf):
    """DRAM bytes per stream-collide launch (mean of an even and an odd step)
    from the committed ncu summary, scaled to nf fluid nodes; None when the
    summary was taken on other kernel sources than the ones built now."""
    path = os.path.join(ROOT, "profiles", f"stream_collide_{layout}_{precision}.md")
    if not os.path.exists(path):
        return None
    src = kernel_source_hash()
    for line in open(path):
        if line.startswith("bench-traffic:"):
            kv = dict(tok.split("=", 1) for tok in line.split()[1:])
            if kv.get("kernel_src") != src:
                return None
            return float(kv["bytes_per_fluid_node"]) * nf
    return None


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(2)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4)
                          if r[3 + k].lower() in ("active", "1")})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def dist_setup(args, backend="nccl"):
    """One process per GPU (torchrun's RANK / LOCAL_RANK / WORLD_SIZE):
    (dist, rank, world size, local rank), or (None, 0, 1, 0) alone.  The
    ranks run independent replicas; the process group carries only the
    timing barrier and the max-reduce of the timed interval."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch
        import torch.distributed as dist

        rank = int(os.environ["RANK"])
        local = int(os.environ.get("LOCAL_RANK", rank))
        if backend == "nccl":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group(backend)
        return dist, rank, ws, local
    return None, 0, 1, 0


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, x, device="cuda"):
    if dist is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, steps, world_size, ms_max):
    """Whole-job throughput in millions of units per second: every rank's
    units over the slowest rank's time (weak scaling, fixed work per rank)."""
    return units_per_rank * steps * world_size / (ms_max * 1e-3) / 1e6


# ------------------------------------------------------------------ oracle

def oracle_sample(mask, seconds=12.0, nz=64):
    """FP64 oracle on a z-slab of the workload (periodic in z), stepped until
    `seconds` of host time have passed; returns (fluid MLUPS, threads, text)."""
    import oracle

    oracle.build()
    oracle.set_threads(os.cpu_count() or 1)
    slab = np.ascontiguousarray(mask[:nz])
    O = oracle.Solver(slab, oracle.rates("B", 1.0), [1e-6, 0.0, 0.0])
    nf = int((slab == 0).sum())
    O.step(1)  # first touch
    steps, t0 = 0, time.perf_counter()
    while True:
        O.step(1)
        steps += 1
        dt = time.perf_counter() - t0
        if dt >= seconds or steps >= 50:
            break
    mlups = nf * steps / dt / 1e6
    text = (f"FP64 oracle, z-slab {mask.shape[2]}x{mask.shape[1]}x{nz} of the workload "
            f"(periodic in z), {steps} steps in {dt:.1f} s")
    return mlups, oracle.get_threads(), text


def oracle_extra(mask):
    """The oracle on one thread (two steps of a 512 x 512 x 8 slab of the
    workload) and, on all host threads, the 32^3 simple-cubic case (r = 12,
    Set E(3/16), tau = 1, F = 1e-6) run to the paper's stopping rule at
    tol 1e-9."""
    import oracle

    from paper_1902_11193_gb300 import geometry

    out = {}
    oracle.set_threads(1)
    slab = np.ascontiguousarray(mask[:8])
    O = oracle.Solver(slab, oracle.rates("B", 1.0), [1e-6, 0.0, 0.0])
    O.step(1)
    t0 = time.perf_counter()
    O.step(2)
    dt = time.perf_counter() - t0
    out["single_thread_MLUPS"] = int((slab == 0).sum()) * 2 / dt / 1e6
    oracle.set_threads(os.cpu_count() or 1)
    m = geometry.sphere_array(32, "sc", r=12)
    O = oracle.Solver(m, oracle.rates("E", 1.0, 3 / 16), [1e-6, 0.0, 0.0])
    t0 = time.perf_counter()
    rc, steps, _ = O.run_to_convergence(1e-9, K=1, max_steps=100000)
    dt = time.perf_counter() - t0
    out["sc32_to_convergence"] = {"steps": steps, "seconds": dt, "threads": oracle.get_threads(),
                                  "fluid_MLUPS": int((m == 0).sum()) * steps / dt / 1e6,
                                  "converged": rc == 0}
    return out


def run_reference(args):
    dist, rank, ws, _ = (None, 0, 1, 0)
    if int(os.environ.get("WORLD_SIZE", "1")) > 1 and int(os.environ.get("RANK", "0")) != 0:
        return
    mask, _ = workload(args.size)
    # each step is a bounded sample: one oracle step on a 512 x 512 x 8 slab
    import oracle

    oracle.build()
    oracle.set_threads(os.cpu_count() or 1)
    slab = np.ascontiguousarray(mask[:8])
    nf = int((slab == 0).sum())
    O = oracle.Solver(slab, oracle.rates("B", 1.0), [1e-6, 0.0, 0.0])
    for _ in range(max(args.warmup, 0)):
        O.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.step(1)
    dt = time.perf_counter() - t0
    mlups = nf * args.steps / dt / 1e6
    line = {
        "impl": "reference", "metric": "fluid MLUPS", "value": mlups, "unit": "fluid MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args),
                   "sample": f"each step: one FP64 oracle step on the {args.size}x{args.size}x8 "
                             "z-slab of the workload (periodic in z)"},
        "cpu_baseline": {"value": mlups, "unit": "fluid MLUPS", "cores": oracle.get_threads(),
                         "kind": "oracle",
                         "sample": f"{args.size}x{args.size}x8 z-slab, {args.steps} steps"},
        "e2e": {"value": mlups, "unit": "fluid MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------- ours

def make_solver(mask, args, layout=None, precision=None, stream=None, max_steps=1_000_000,
                collision="auto"):
    from paper_1902_11193_gb300 import lbm

    return lbm.LBMSolver(mask, "B", 1.0, force=(1e-6, 0.0, 0.0),
                         precision=precision or args.precision, layout=layout or args.layout,
                         check_interval=100, max_steps=max_steps, stream=stream,
                         block_size=args.block_size, collision=collision)


def time_production_loop(S, steps, stream):
    """Events around lbm_run_to_convergence(tol=0) capped at `steps`."""
    import torch

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    rc, taken = S.run_to_convergence(0.0)
    e1.record(stream)
    torch.cuda.synchronize()
    assert taken == steps, (rc, taken)
    return e0.elapsed_time(e1)


def time_kernel_launches(S, n, stream, split=False):
    """Average device time of one plain stream-collide launch (events between
    consecutive launches on the launching stream).  split=True also returns
    the mean times of the even-step and odd-step launches (AA patterns: two
    kernels; AB: the same kernel on both parities)."""
    import torch

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(n + 1)]
    torch.cuda.synchronize()
    p0 = S.steps % 2
    ev[0].record(stream)
    for i in range(n):
        S.step(1)
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    d = np.array([ev[i].elapsed_time(ev[i + 1]) for i in range(n)])
    if not split:
        return float(np.mean(d)), float(np.min(d))
    par = (p0 + np.arange(n)) % 2
    return (float(np.mean(d)), float(np.min(d)), float(np.mean(d[par == 0])),
            float(np.mean(d[par == 1])))


# kernels of each layout's plain stream-collide launches (even step, odd step)
STEP_KERNELS = {
    ("sparse", "fp32"): ("k_sparse_even_x2", "k_sparse_odd_l"),
    ("sparse", "fp16"): ("k_sparse_even_h4", "k_sparse_odd_l"),
    ("sparse", "fp64"): ("k_sparse", "k_sparse_odd_t"),
    ("aa", "fp32"): ("k_aa<even>", "k_aa<odd>"), ("aa", "fp16"): ("k_aa<even>", "k_aa<odd>"),
    ("aa", "fp64"): ("k_aa<even>", "k_aa<odd>"),
}


def collision_form(set_, collision):
    """The collision the kernels run: the link-basis TRT where the rates have
    one even and one odd value (Sets B, E, SRT) unless the MRT is forced."""
    return "trt" if collision == "auto" and set_ in ("B", "E", "SRT") else "mrt"


def run_ours(args):
    import torch

    from paper_1902_11193_gb300 import lbm

    dist, rank, ws, local = dist_setup(args)
    torch.cuda.set_device(local)
    # a stream of our own (the default stream's handle is 0, which the library
    # would replace by a stream of its own), current for torch's events too
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    mask, nspheres = workload(args.size)
    nf = int((mask == 0).sum())
    N = mask.size
    warm = max(args.warmup, 3)

    S = make_solver(mask, args, stream=stream, max_steps=args.steps)
    l0 = S.kernel_launches
    S.step(warm)
    torch.cuda.synchronize()
    barrier(dist)
    launches0 = S.kernel_launches
    with ClockSampler(local) as clk:
        ms = time_production_loop(S, args.steps, stream)
    launches = S.kernel_launches - launches0
    k_fp = S.permeability()
    ms = max_over_ranks(dist, ms)
    value = job_throughput(nf, args.steps, ws, ms)
    # the stream-collide launches alone: per-launch event timing on their
    # stream, even and odd steps apart
    kmean, kmin, keven, kodd = time_kernel_launches(S, 50, stream, split=True)
    S.close()
    del S

    peak, peak_kind = load_peaks()
    bpu = BYTES_PER_UPDATE[args.precision]
    achieved = bpu * nf / (kmean * 1e-3) / 1e9
    traffic = measured_traffic(args.layout, args.precision, nf)
    kern = STEP_KERNELS.get((args.layout, args.precision), ("k_ab", "k_ab"))
    if (args.layout, args.precision) == ("sparse", "fp16"):
        # plain FP16 even steps pair adjacent nodes per 32-bit word when N_f is even
        kern = ("k_sparse_even_p2" if nf % 2 == 0 else "k_sparse_even_h4", kern[1])

    out = {
        "metric": "fluid MLUPS", "value": value, "unit": "fluid MLUPS", "n_gpus": ws,
        "steps": args.steps, "warmup": warm, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp16": "f32 (f16 storage)", "fp64": "f64"}[args.precision],
        "data": "synthetic",
        "config": {"workload": workload_name(args), "nodes": N, "fluid_nodes": nf,
                   "spheres": nspheres, "l2": "inputs larger than L2 "
                   f"({bpu // 2 * (nf if args.layout == 'sparse' else N) / 1e9:.1f} GB of "
                   "populations), no flush", "parallelism": f"replicas x{ws}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": f"stream-collide {args.layout} {args.precision}",
                     "algorithmic_bytes_per_launch": bpu * nf,
                     "launch_ms_mean": kmean, "launch_ms_min": kmin,
                     "launch_ms_even": keven, "launch_ms_odd": kodd,
                     "frac_even": bpu * nf / (keven * 1e-3) / 1e9 / peak,
                     "frac_odd": bpu * nf / (kodd * 1e-3) / 1e9 / peak,
                     "kernel_even": kern[0], "kernel_odd": kern[1],
                     "dominant": kern[1] if kodd >= keven else kern[0],
                     "frac_dominant": bpu * nf / (max(kodd, keven) * 1e-3) / 1e9 / peak,
                     "collision": collision_form("B", "auto"),
                     "frac_definition": "frac: algorithmic bytes per launch over the mean "
                                        "launch time of an even and an odd step (one AA "
                                        "step pair); frac_even, frac_odd, frac_dominant: "
                                        "per kernel",
                     "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)"},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "permeability_lu": float(k_fp[0]),
    }

    if rank == 0 and not args.no_extra:
        # the same workload with the moment-space MRT collision forced
        S2 = make_solver(mask, args, stream=stream, max_steps=200, collision="mrt")
        S2.step(warm)
        m2 = time_production_loop(S2, 200, stream)
        km, _, ke, ko = time_kernel_launches(S2, 50, stream, split=True)
        out["mrt"] = {"collision": "mrt", "fluid_MLUPS": nf * 200 / (m2 * 1e-3) / 1e6,
                      "launch_ms_even": ke, "launch_ms_odd": ko,
                      "frac": bpu * nf / (km * 1e-3) / 1e9 / peak,
                      "frac_even": bpu * nf / (ke * 1e-3) / 1e9 / peak,
                      "frac_odd": bpu * nf / (ko * 1e-3) / 1e9 / peak}
        S2.close()
        out["layouts"] = {}
        for lay in ("aa", "sparse", "ab"):
            if lay == args.layout:
                continue
            S2 = make_solver(mask, args, layout=lay, stream=stream, max_steps=200)
            S2.step(warm)
            m2 = time_production_loop(S2, 200, stream)
            out["layouts"][lay] = nf * 200 / (m2 * 1e-3) / 1e6
            S2.close()
        out["perm_rel_err"] = permeability_errors(args, stream)

    if rank == 0 and not args.no_e2e:
        out["e2e"] = e2e_run(mask, args, stream)

    if rank == 0 and args.sweep != "none":
        out["sweep"] = sweep_run(args, stream)
    if rank == 0 and args.adjoint:
        out["adjoint"] = adjoint_run(args, stream)
    if rank == 0 and args.large:
        out["large"] = large_run(args, stream)
    if rank == 0 and args.channels != "none":
        out["channels"] = channels_run(args, stream)

    if rank == 0 and not args.no_cpu_baseline:
        v, cores, text = oracle_sample(mask)
        out["cpu_baseline"] = {"value": v, "unit": "fluid MLUPS", "cores": cores,
                               "kind": "oracle", "sample": text}
        out["cpu_baseline"].update(oracle_extra(mask))
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def permeability_errors(args, stream):
    """Permeability of the 32^3 simple-cubic cell (sphere r = 12, Set E(3/16),
    tau = 1, F = 1e-6) at the FP64 oracle's stop step, per precision, against
    the stored oracle value (tests/golden/oracle_config1.txt)."""
    from paper_1902_11193_gb300 import geometry, lbm

    path = os.path.join(ROOT, "tests", "golden", "oracle_config1.txt")
    row = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")][0]
    steps, k_ora = int(row[0]), float(row[1])
    mask = geometry.sphere_array(32, "sc", r=12)
    res = {"workload": "32^3 SC r=12, Set E(3/16), tau=1, F=1e-6, at the oracle's stop step "
                       f"{steps} (tol 1e-9)", "k_oracle": k_ora}
    for prec, lay in (("fp64", "ab"), ("fp32", "aa"), ("fp32", "sparse"), ("fp16", "sparse")):
        S = lbm.LBMSolver(mask, "E", 1.0, 3 / 16, (1e-6, 0, 0), precision=prec, layout=lay,
                          stream=stream)
        S.step(steps)
        k = S.permeability()[0]
        res[f"{prec}_{lay}"] = abs(k - k_ora) / abs(k_ora)
        S.close()
    return res


def e2e_run(mask, args, stream):
    """The whole job through the C ABI from host memory: lbm_create from the
    host mask (H2D), the production loop, lbm_permeability (D2H)."""
    import torch

    steps = args.steps
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    S = make_solver(mask, args, stream=stream, max_steps=steps)
    S.run_to_convergence(0.0)
    k = S.permeability()
    t1 = time.perf_counter()
    S.close()
    nf = int((mask == 0).sum())
    chunks = (steps + 99) // 100
    return {"value": nf * steps / (t1 - t0) / 1e6, "unit": "fluid MLUPS",
            "h2d_bytes_per_step": mask.nbytes / steps,
            "d2h_bytes_per_step": (chunks * (2 * 3 * 8 + 4) + 3 * 8) / steps,
            "wall_s": t1 - t0, "permeability_lu": float(k[0]),
            "includes": "lbm_create (mask upload, link tables, allocation), the production "
                        "loop, lbm_permeability"}


SWEEP_TAUS = (0.6, 0.8, 1.0, 1.15, 1.3, 1.6, 2.0)
SWEEP_SETS = (("A", 3 / 16), ("B", 3 / 16), ("C", 3 / 16), ("D", 3 / 16), ("E", 1 / 64),
              ("E", 3 / 16), ("E", 3 / 8))


def sweep_lattices(kind):
    """The parameter study of Secs. 4.1-4.3 on sphere arrays: SC/BCC/FCC cells
    at solid fractions 0.1-0.5 and edges 16/32/64/96 x Sets A-E x 7 taus
    ("full", 2940 lattices), or a seeded subset of it (edges 16/32, three
    fractions, three taus, all seven rate sets: 378 lattices)."""
    from paper_1902_11193_gb300 import geometry

    if kind == "full":
        edges, fracs, taus = (16, 32, 64, 96), (0.1, 0.2, 0.3, 0.4, 0.5), SWEEP_TAUS
    else:
        edges, fracs, taus = (16, 32), (0.1, 0.3, 0.5), (0.6, 1.0, 1.6)
    lats = []
    for arr in ("sc", "bcc", "fcc"):
        for L in edges:
            for c in fracs:
                m = geometry.sphere_array(L, arr, c=c)
                for st, lam in SWEEP_SETS:
                    for tau in taus:
                        lats.append(dict(mask=m, set_=st, tau=tau, Lambda=lam,
                                         force=(1e-6, 0.0, 0.0)))
    return lats


def sweep_run(args, stream):
    """Converges every lattice of the sweep (paper's rule, tol 1e-6 on k) in
    one batch, then the same lattices one by one through lbm_run_to_convergence;
    wall time of each, launches of each."""
    import torch

    from paper_1902_11193_gb300 import lbm

    lats = sweep_lattices(args.sweep)
    K = 100
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    B = lbm.LBMBatch(lats, precision="fp32", check_interval=K, max_steps=200000, stream=stream)
    t1 = time.perf_counter()
    steps, status = B.run(1e-6)
    kb = B.permeability()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    lay, npt = B.config()
    blaunch = B.kernel_launches
    chunks = B.schedule_counts()
    B.close()
    t3 = time.perf_counter()
    ks, seq_launches, seq_steps = [], 0, []
    by_edge = {}
    for l, layout in zip(lats, lay):
        ts = time.perf_counter()
        S = lbm.LBMSolver(l["mask"], l["set_"], l["tau"], l["Lambda"], l["force"],
                          precision="fp32", layout=["ab", "aa", "sparse"][layout],
                          check_interval=K, max_steps=200000, stream=stream)
        rc, st = S.run_to_convergence(1e-6)
        ks.append(S.converged_permeability())  # k of the measure the rule stopped on
        seq_launches += S.kernel_launches
        seq_steps.append(st)
        S.close()
        e = str(l["mask"].shape[0])
        by_edge[e] = by_edge.get(e, 0.0) + time.perf_counter() - ts
    torch.cuda.synchronize()
    t4 = time.perf_counter()
    fluid = np.array([int((l["mask"] == 0).sum()) for l in lats])
    updates = float(np.sum(fluid * steps))
    return {"lattices": len(lats), "kind": args.sweep, "tol": 1e-6, "check_interval": K,
            "converged": int(np.sum(status == 0)), "steps_total": int(steps.sum()),
            "batched_s": t2 - t1, "batched_setup_s": t1 - t0, "sequential_s": t4 - t3,
            "speedup": (t4 - t3) / (t2 - t1),
            "batched_fluid_MLUPS": updates / (t2 - t1) / 1e6,
            "sequential_fluid_MLUPS": float(np.sum(fluid * np.array(seq_steps))) / (t4 - t3) / 1e6,
            "batched_launches": blaunch, "sequential_launches": seq_launches,
            "same_steps": bool(np.array_equal(steps, np.array(seq_steps))),
            "max_k_diff": float(np.max(np.abs(np.array(ks)[:, 0] - kb[:, 0]))),  # driven (x) component
            "k_bitwise_equal": bool(np.array_equal(np.array(ks)[:, 0], kb[:, 0])),
            "layouts": {"aa": int(np.sum(lay == 1)), "sparse": int(np.sum(lay == 2)),
                        "npt2": int(np.sum(npt == 2)), "alone": int(np.sum(npt == 0))},
            "chunks": {"stepwise": chunks[0], "persistent": chunks[1]},
            "sequential_s_by_edge": by_edge}


def adjoint_grads(S, g, set_, lam, tau, F):
    """Normalised gradients theta (dk/dtheta) / k of one steady adjoint."""
    k = g["k"]
    out = {"k": k, "tau_dk_dtau_over_k": g["dtau"] * tau / k,
           "F_dk_dF_over_k": g["dF"][0] * F / k, "adjoint_iterations": g["iterations"],
           "adjoint_residual": g["residual"]}
    if set_ == "D":  # two magic parameters, 3/16 for s_q and 3/8 for s_m at every tau
        out["Lq_dk_dLq_over_k"] = g["dLambda_q"] * (3 / 16) / k
        out["Lm_dk_dLm_over_k"] = g["dLambda_m"] * (3 / 8) / k
    else:  # B (= E(3/16)) and E: one magic parameter for both odd rates
        out["L_dk_dL_over_k"] = g["dLambda"] * lam / k
    return out


def adjoint_run(args, stream):
    """Steady adjoint on a Boolean medium (r = 6, porosity 0.35, edge
    --adjoint-size, 128 by default): for Sets B, D, E(3/16), E(3/8) at
    tau = 0.8, 1.0, 1.3, the FP32 forward to the two-step-mean rule, then
    lbm_adjoint; gradients normalised.  Then the transient adjoint of Set D
    at tau = 1 over the same number of steps."""
    import torch

    from paper_1902_11193_gb300 import geometry, lbm

    L = args.adjoint_size
    F = 1e-6
    mask, _ = geometry.boolean(L, 6, 0.35, seed=1902_11193 + 4)
    nf = int((mask == 0).sum())
    res = {"workload": f"boolean-{L}^3 r=6 porosity=0.35, F=1e-6 x, fp32 sparse, two-step-mean "
                       "stopping rule (tol 1e-8), adjoint tol 1e-6; sets "
                       f"{args.adjoint_sets} x tau {args.adjoint_taus}", "grid": []}
    steps_d1 = None
    t_fwd = t_adj = 0.0
    iters = 0
    sets = []
    for tok in args.adjoint_sets.split(","):
        if tok.startswith("E"):
            num, den = tok[1:].split("/")
            sets.append(("E", float(num) / float(den)))
        else:
            sets.append((tok, 3 / 16))
    taus = tuple(float(t) for t in args.adjoint_taus.split(","))
    for set_, lam in sets:
        for tau in taus:
            S = lbm.LBMSolver(mask, set_, tau, lam, force=(F, 0, 0), precision="fp32",
                              layout="sparse", check_interval=100, stream=stream, stop_rule=1,
                              max_steps=400000)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc, steps = S.run_to_convergence(1e-8, raise_on_failure=False)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            row = {"set": set_ if set_ != "E" else f"E({lam:g})", "tau": tau,
                   "forward_status": rc, "forward_steps": steps}
            if rc == 0:
                g = S.adjoint(1e-6, max_iter=400000)
                torch.cuda.synchronize()
                t2 = time.perf_counter()
                row.update(adjoint_grads(S, g, set_, lam, tau, F))
                t_fwd += t1 - t0
                t_adj += t2 - t1
                iters += g["iterations"]
                if set_ == "D" and tau == 1.0:
                    steps_d1 = steps
            res["grid"].append(row)
            S.close()
    res["forward_s_total"] = t_fwd
    res["adjoint_s_total"] = t_adj
    res["adjoint_fluid_MLUPS"] = nf * iters / t_adj / 1e6 if t_adj > 0 else None
    if steps_d1 is None or args.no_transient:
        return res
    # transient adjoint: the gradient of k after the same number of steps
    # from rest, by a checkpointed reverse sweep
    T = lbm.LBMSolver(mask, "D", 1.0, force=(F, 0, 0), precision="fp32", layout="sparse",
                      stream=stream)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    gt = T.adjoint_transient(steps_d1)
    torch.cuda.synchronize()
    t4 = time.perf_counter()
    res["transient"] = {
        "set": "D", "tau": 1.0, "steps": steps_d1, "wall_s": t4 - t3,
        # forward sweep, recomputation of every segment, adjoint step: three passes
        "fluid_MLUPS_per_pass": 3 * nf * steps_d1 / (t4 - t3) / 1e6,
        "k": gt["k"], "tau_dk_dtau_over_k": gt["dtau"] * 1.0 / gt["k"],
        "Lq_dk_dLq_over_k": gt["dLambda_q"] * (3 / 16) / gt["k"],
        "Lm_dk_dLm_over_k": gt["dLambda_m"] * (3 / 8) / gt["k"]}
    T.close()
    return res


CHANNEL_TAUS = (0.6, 0.8, 1.0, 1.15, 1.3, 1.6, 2.0)
CHANNEL_SETS = (("SRT", 3 / 16), ("A", 3 / 16), ("B", 3 / 16), ("C", 3 / 16), ("D", 3 / 16),
                ("E", 1 / 64), ("E", 3 / 16), ("E", 3 / 8))


def channel_geometries(kind):
    """Circular bores of diameter D in an L^2 section (porosity 0.196) and the
    equilateral triangle of side 200 in 256^2, as one-voxel periodic slabs, with
    the references k = pi R^4 / (8 A) and sqrt(3) l^4 / (320 A)."""
    from paper_1902_11193_gb300 import geometry

    circles = [(32, 128), (64, 256)] + ([(128, 512)] if kind == "full" else [])
    out = [(f"circle D={D} in {L}^2", geometry.pipe(D, L), np.pi * (D / 2) ** 4 / (8 * L * L))
           for D, L in circles]
    if kind == "full":
        out.append(("triangle l=200 in 256^2", geometry.triangle(200, 256),
                    np.sqrt(3) * 200.0**4 / (320 * 256 * 256)))
    return out


def channels_run(args, stream):
    """The paper's channel study (Secs. 4.1-4.2) in one batch: every geometry
    x rate set x tau, converged (K = 100, tol 1e-10 on the per-check relative
    change of U), then k / k_ref per geometry and set: mean over tau and the
    relative spread (max - min) / mean; plus the resolution series of circular
    bores D = 16, 24, 36, 48 in a 64^2 section (SRT, Set B, Set E(3/8), tau = 1)."""
    import torch

    from paper_1902_11193_gb300 import geometry, lbm

    geoms = channel_geometries(args.channels)
    lats, keys = [], []
    for gname, m, kref in geoms:
        for st, lam in CHANNEL_SETS:
            for tau in CHANNEL_TAUS:
                lats.append(dict(mask=m, set_=st, tau=tau, Lambda=lam, force=(1e-6, 0.0, 0.0)))
                keys.append((gname, st, lam, tau, kref))
    series = []
    for D in (16, 24, 36, 48):
        m = geometry.pipe(D, 64)
        for st, lam in (("SRT", 3 / 16), ("B", 3 / 16), ("E", 3 / 8)):
            lats.append(dict(mask=m, set_=st, tau=1.0, Lambda=lam, force=(1e-6, 0.0, 0.0)))
            keys.append((f"series D={D}", st, lam, 1.0, np.pi * (D / 2) ** 4 / (8 * 64 * 64)))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    B = lbm.LBMBatch(lats, precision="fp64", check_interval=100, max_steps=2_000_000, stream=stream)
    steps, status = B.run(1e-10)
    k = B.permeability()[:, 0]
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    lay, _ = B.config()
    B.close()
    fluid = np.array([int((l["mask"] == 0).sum()) for l in lats])
    res = {"workload": "one-voxel periodic slabs, F = 1e-6 along the bore, fp64 batch, "
                       "K = 100, tol 1e-10; sets SRT, A, B, C, D, E(1/64, 3/16, 3/8); "
                       "tau " + ", ".join(str(t) for t in CHANNEL_TAUS),
           "lattices": len(lats), "converged": int(np.sum(status == 0)),
           "steps_total": int(steps.sum()), "steps_max": int(steps.max()), "wall_s": t1 - t0,
           "fluid_MLUPS": float(np.sum(fluid * steps)) / (t1 - t0) / 1e6,
           "layouts": {"aa": int(np.sum(lay == 1)), "sparse": int(np.sum(lay == 2))},
           "geometries": {}}
    i = 0
    for gname, _, _ in geoms:
        g = {}
        for st, lam in CHANNEL_SETS:
            r = k[i:i + len(CHANNEL_TAUS)] / keys[i][4]
            st_steps = steps[i:i + len(CHANNEL_TAUS)]
            g[f"{st}({lam:g})" if st == "E" else st] = {
                "k_over_kref_mean": float(np.mean(r)), "spread": float(np.ptp(r) / np.mean(r)),
                "steps_tau_min": int(st_steps[0]), "steps_tau_max": int(st_steps[-1])}
            i += len(CHANNEL_TAUS)
        res["geometries"][gname] = g
    ser = {}
    for j in range(i, len(lats)):
        gname, st, lam, _, kref = keys[j]
        ser.setdefault(gname, {})[f"{st}({lam:g})" if st == "E" else st] = float(k[j] / kref)
    res["resolution_series_k_over_kref"] = ser
    return res


def large_run(args, stream):
    """1024^3 Boolean medium (r = 8, porosity 0.20), Set D, tau = 1, sparse
    layout: FP32 vs FP16 storage (FP32 arithmetic), per-launch timing of 40
    steps after warm-up, and the relative difference of the mean velocity
    between the two storages after the same number of steps."""
    import torch

    from paper_1902_11193_gb300 import geometry, lbm

    t0 = time.perf_counter()
    mask, ns = geometry.boolean(1024, 8, 0.20, seed=1902_11193 + 5)
    tgen = time.perf_counter() - t0
    nf = int((mask == 0).sum())
    res = {"workload": "boolean-1024^3 r=8 porosity=0.20, Set D tau=1, F=1e-6, sparse",
           "fluid_nodes": nf, "spheres": ns, "mask_gen_s": tgen}
    U = {}
    peak, _ = load_peaks()
    for prec in ("fp32", "fp16"):
        S = lbm.LBMSolver(mask, "D", 1.0, force=(1e-6, 0, 0), precision=prec, layout="sparse",
                          stream=stream)
        S.step(10)
        kmean, kmin = time_kernel_launches(S, 40, stream)
        U[prec] = S.mean_velocity()[0]
        mlups = nf / (kmean * 1e-3) / 1e6
        res[prec] = {"fluid_MLUPS": mlups, "launch_ms_mean": kmean,
                     "hbm_frac_algorithmic": BYTES_PER_UPDATE[prec] * nf / (kmean * 1e-3) / 1e9 / peak}
        S.close()
        torch.cuda.synchronize()
    res["fp16_vs_fp32_mean_velocity_rel_diff_after_50_steps"] = abs(U["fp16"] - U["fp32"]) / abs(U["fp32"])
    res["k_error"] = reduced_precision_k_errors(stream)
    return res


def reduced_precision_k_errors(stream, L=256):
    """Permeability of a converged sample with the 1024^3 workload's recipe
    (Boolean medium, r = 8, porosity 0.20, Set D, tau = 1, F = 1e-6, sparse),
    at edge L: FP64 to the two-step-mean rule (tol 1e-8, K = 100), then FP32
    and FP16 storage for the same number of steps; each k (the two-step mean
    of the last chunk) against the FP64 one."""
    import torch

    from paper_1902_11193_gb300 import geometry, lbm

    mask, _ = geometry.boolean(L, 8, 0.20, seed=1902_11193 + 5)
    kw = dict(force=(1e-6, 0, 0), layout="sparse", check_interval=100, stream=stream,
              stop_rule=1)
    t0 = time.perf_counter()
    S = lbm.LBMSolver(mask, "D", 1.0, precision="fp64", max_steps=400000, **kw)
    rc, steps = S.run_to_convergence(1e-8, raise_on_failure=False)
    k64 = S.converged_permeability()[0]
    S.close()
    res = {"workload": f"boolean-{L}^3 r=8 porosity=0.20 seed={1902_11193 + 5}, Set D tau=1, "
                       "F=1e-6, sparse; FP64 to tol 1e-8 (two-step mean, K=100), FP32 and "
                       "FP16 storage for the same steps",
           "fluid_nodes": int((mask == 0).sum()), "fp64_status": rc, "steps": steps,
           "k_fp64": k64}
    for prec in ("fp32", "fp16"):
        S = lbm.LBMSolver(mask, "D", 1.0, precision=prec, max_steps=steps, **kw)
        S.run_to_convergence(0.0, raise_on_failure=False)
        k = S.converged_permeability()[0]
        res[f"k_{prec}"] = k
        res[f"{prec}_rel_err"] = abs(k - k64) / abs(k64)
        S.close()
    torch.cuda.synchronize()
    res["wall_s"] = time.perf_counter() - t0
    return res


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
