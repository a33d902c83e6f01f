"""Every kernel family of the library on tiny lattices, for the bounds-check
build (test code only).

`run_cases()` runs ragged 4^3-8^3 lattices with fluid on every face through
the stream-collide kernels of the three layouts and three storage
precisions (plain and measuring steps, 32- and 64-bit offsets), the state
readers and writers, the steady and transient adjoints, the batched
persistent kernel, the bounded-domain and full-way bounceback kernels and
the allocation-free mean velocity.  It returns every result array and the
device flags each context reported.  As a script,

    python tests/bounds_cases.py LIBRARY OUT.npz

it loads the given library build instead of the package's own one and
writes the results to OUT.npz.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
F3 = (1e-4, 2e-5, -1e-5)


def _masks():
    from paper_1902_11193_gb300 import geometry

    out = {}
    for i, dims in enumerate(((5, 6, 7), (8, 4, 6), (4, 4, 4), (7, 5, 8))):
        m = geometry.random_mask(dims[::-1], 0.3, seed=40 + i)
        # fluid on every face: the wrapped upstream indices are all exercised
        m[0, :, :] = m[-1, :, :] = 0
        m[:, 0, :] = m[:, -1, :] = 0
        m[:, :, 0] = m[:, :, -1] = 0
        m[1, 1, 1] = 1  # and some solid next to them
        out[f"m{i}"] = m
    return out


def _random_state(mask, seed):
    rng = np.random.default_rng(seed)
    f = W[:, None, None, None] * (1 + 1e-2 * rng.standard_normal((19,) + mask.shape))
    f[:, mask == 1] = W[:, None]
    return f


def run_cases():
    import torch

    from paper_1902_11193_gb300 import lbm

    res, flags = {}, {}

    def note(key, S):
        flags[key] = S.device_flags()

    masks = _masks()
    for mname, mask in masks.items():
        nodes = np.flatnonzero(mask.reshape(-1) == 0)[::3].astype(np.int64)
        for layout in ("ab", "aa", "sparse"):
            for prec in ("fp64", "fp32", "fp16"):
                for width in ((0, 64) if layout == "sparse" else (0,)):
                    key = f"{mname}_{layout}_{prec}_w{width}"
                    S = lbm.LBMSolver(mask, "D", 0.9, force=F3, precision=prec, layout=layout,
                                      check_interval=4, max_steps=11, index_width=width)
                    S.set_populations(_random_state(mask, 5))
                    S.step(7)
                    res[key + "_f"] = S.get_populations()
                    res[key + "_u"] = S.velocity()
                    res[key + "_U"] = S.mean_velocity()
                    res[key + "_at"] = S.get_populations_at(nodes)
                    S.run_to_convergence(0.0, raise_on_failure=False)  # measuring steps
                    res[key + "_conv"] = S.converged_velocity()
                    note(key, S)
                    S.close()
        # steady and transient adjoints, two-step-mean rule
        for layout in ("ab", "aa", "sparse"):
            for prec in ("fp64", "fp32"):
                key = f"{mname}_adj_{layout}_{prec}"
                S = lbm.LBMSolver(mask, "B", 0.9, force=(1e-5, 0, 0), precision=prec,
                                  layout=layout, check_interval=10, stop_rule=1, max_steps=20000)
                rc, _ = S.run_to_convergence(1e-9 if prec == "fp64" else 1e-6,
                                             raise_on_failure=False)
                if rc == 0:
                    g = S.adjoint(1e-10 if prec == "fp64" else 1e-5, max_iter=20000)
                    res[key + "_g"] = np.array([g["dtau"], g["dLambda"], g["dF"][0]])
                gt = S.adjoint_transient(5)
                res[key + "_gt"] = np.array([gt["dtau"], gt["dLambda"], gt["dF"][0]])
                note(key, S)
                S.close()
        # bounded domains and full-way bounceback (two-array layout)
        for prec in ("fp64", "fp32"):
            key = f"{mname}_bounded_{prec}"
            S = lbm.LBMSolver(mask, "C", 0.8, force=(0, 0, 0), precision=prec, layout="ab",
                              pressure=(1.001, 0.999), symmetry="yz")
            S.step(6)
            res[key + "_u"] = S.velocity()
            res[key + "_U"] = S.mean_velocity()
            note(key, S)
            S.close()
            key = f"{mname}_fullway_{prec}"
            S = lbm.LBMSolver(mask, "A", 0.8, force=F3, precision=prec, layout="ab",
                              bounceback="fullway")
            S.step(6)
            res[key + "_u"] = S.velocity()
            note(key, S)
            S.close()
        # the allocation-free mean velocity of an FP64 two-array state
        S = lbm.LBMSolver(mask, "D", 0.9, force=F3, precision="fp64", layout="ab")
        S.step(5)
        g = torch.from_numpy(np.ascontiguousarray(S.get_populations() - W[:, None, None, None])).cuda()
        m = torch.from_numpy(mask).cuda()
        U = torch.zeros(3, dtype=torch.float64, device="cuda")
        rc = lbm.lib().lbm_mean_velocity_noalloc(
            g.data_ptr(), m.data_ptr(), np.array(mask.shape[::-1], np.int32),
            np.ascontiguousarray(F3, np.float64), U.data_ptr(),
            torch.cuda.current_stream().cuda_stream)
        assert rc == 0
        torch.cuda.synchronize()
        res[f"{mname}_noalloc_U"] = U.cpu().numpy()
        S.close()
    # the batched persistent kernel: every layout and units-per-thread choice
    lats = [dict(mask=m, set_=st, tau=t, Lambda=3 / 16, force=(1e-5, 0, 0))
            for m in masks.values() for st, t in (("B", 0.9), ("D", 1.2))]
    for prec in ("fp32", "fp64"):
        for layout in ("aa", "sparse"):
            for npt in (1, 2):
                B = lbm.LBMBatch(lats, precision=prec, layout=layout, nodes_per_thread=npt,
                                 check_interval=5, max_steps=13, solo="never")
                B.run(0.0, raise_on_failure=False)
                res[f"batch_{prec}_{layout}_{npt}"] = B.mean_velocity()
                for i in range(len(lats)):
                    flags[f"batch_{prec}_{layout}_{npt}_{i}"] = B.lattice(i).device_flags()
                B.close()
    return res, flags


def main():
    lib_path, out = sys.argv[1], sys.argv[2]
    from paper_1902_11193_gb300 import _build

    _build.LBM_SO = lib_path
    res, flags = run_cases()
    np.savez(out, **res, **{"flags__" + k: np.array(v) for k, v in flags.items()})


if __name__ == "__main__":
    main()
