"""The link-basis TRT collision on the CUDA path (Sec. 2.2).

Where the rates have one even and one odd value (Sets B, E, SRT) the
kernels collide in link form by default; collision="mrt" forces the
moment-space form.  Both are the same collision: they agree with each other
and with the FP64 oracle's MRT to rounding, and lattices whose rates are not
of that shape (Set D) run the MRT either way, bit for bit.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

F3 = (1e-4, 2e-5, -1e-5)


@pytest.fixture(scope="module")
def L():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_11193_gb300 import lbm

    lbm.lib()
    return lbm


@pytest.mark.parametrize("st,tau,lam", [("B", 0.7, 3 / 16), ("E", 1.3, 3 / 8), ("SRT", 0.9, 3 / 16)])
@pytest.mark.parametrize("layout", ["ab", "aa", "sparse"])
def test_trt_equals_mrt_and_oracle(L, ora, geom, st, tau, lam, layout):
    mask = geom.boolean(24, 4, 0.45, seed=1902_11193 + 11)[0]
    O = ora.Solver(mask, ora.rates(st, tau, lam), F3)
    T = L.LBMSolver(mask, st, tau, lam, F3, precision="fp64", layout=layout)
    M = L.LBMSolver(mask, st, tau, lam, F3, precision="fp64", layout=layout, collision="mrt")
    for n in (1, 7, 50):
        O.step(n - O.steps)
        T.step(n - T.steps)
        M.step(n - M.steps)
        uo, ut, um = O.velocity(), T.velocity(), M.velocity()
        scale = np.abs(uo).max()
        assert np.abs(ut - um).max() <= 1e-13 * scale + 1e-16
        assert np.abs(ut - uo).max() <= 1e-12 * scale + 1e-15
    T.close()
    M.close()


def test_mrt_only_sets_ignore_the_switch(L, geom):
    mask = geom.sphere_array(16, "bcc", c=0.3)
    a = L.LBMSolver(mask, "D", 1.1, force=F3, precision="fp32", layout="sparse")
    b = L.LBMSolver(mask, "D", 1.1, force=F3, precision="fp32", layout="sparse", collision="mrt")
    a.step(40)
    b.step(40)
    assert np.array_equal(a.get_populations(), b.get_populations())


def test_trt_fp32_permeability(L, ora, geom):
    mask = geom.sphere_array(20, "fcc", c=0.3)
    tau = 0.8
    O = ora.Solver(mask, ora.rates("B", tau), [1e-6, 0, 0])
    rc, steps, U = O.run_to_convergence(1e-9, K=20, max_steps=200000)
    assert rc == 0
    S = L.LBMSolver(mask, "B", tau, force=(1e-6, 0, 0), precision="fp32", layout="sparse",
                    check_interval=20)
    S.step(steps)
    k = S.permeability()[0]
    ko = (tau - 0.5) / 3 * U[0] / 1e-6
    assert abs(k / ko - 1) <= 1e-5
