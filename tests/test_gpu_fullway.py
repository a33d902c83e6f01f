"""Full-way bounceback (the paper's boundary scheme, Sec. 3) on the CUDA path.

The AB kernel with full-way bounceback against the FP64 oracle's full-way
solver at equal step counts (velocity field and fluid-node populations),
converged k equal to the halfway-bounceback k, and the option's contract:
AB only, no adjoint, link counts of the mask, checkpoints keep the scheme.
"""
import numpy as np
import pytest

from gpu_util import W, dev_err

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


def _masks(geom):
    return {
        "sc32": geom.sphere_array(32, "sc", r=12),
        "boolean32": geom.boolean(32, 4, 0.4, seed=1902_11193 + 7)[0],
        "random_ragged": geom.random_mask((20, 17, 13), 0.3, seed=11),
    }


@pytest.mark.parametrize("name", ["sc32", "boolean32", "random_ragged"])
def test_fullway_fp64_matches_oracle(L, ora, geom, name):
    mask = _masks(geom)[name]
    st, tau = "D", 0.8
    O = ora.Solver(mask, ora.rates(st, tau), F3, bounceback="fullway")
    S = L.LBMSolver(mask, st, tau, force=F3, precision="fp64", layout="ab", bounceback="fullway")
    for n in (1, 6, 40):
        O.step(n - O.steps)
        S.step(n - S.steps)
        uo, ug = O.velocity(), S.velocity()
        assert np.abs(ug - uo).max() <= 1e-12 * np.abs(uo).max() + 1e-15
        fo, fg = O.get_f(), S.get_populations()
        fluid = mask == 0
        assert dev_err(fg[:, fluid], fo[:, fluid], W[:, None]) <= 1e-11
        Uo = O.mean_velocity()
        assert np.abs(S.mean_velocity() - Uo).max() <= 1e-12 * np.abs(Uo).max() + 1e-15
    S.close()


def test_fullway_converged_k_equals_halfway(L, geom):
    mask = geom.sphere_array(24, "bcc", c=0.3)
    k, early = {}, {}
    for bb in ("halfway", "fullway"):
        S = L.LBMSolver(mask, "D", 1.2, force=(1e-6, 0, 0), precision="fp64", layout="ab",
                        check_interval=10, bounceback=bb)
        S.step(10)
        early[bb] = S.mean_velocity()[0]
        rc, _ = S.run_to_convergence(1e-13)
        assert rc == 0
        k[bb] = S.converged_permeability()[0]
        S.close()
    assert abs(k["fullway"] / k["halfway"] - 1) <= 1e-9
    assert abs(early["fullway"] / early["halfway"] - 1) > 1e-3


def test_fullway_fp32_permeability(L, ora, geom):
    mask = geom.sphere_array(16, "fcc", c=0.3)
    tau = 1.0
    O = ora.Solver(mask, ora.rates("B", tau), [1e-6, 0, 0], bounceback="fullway")
    rc, steps, U = O.run_to_convergence(1e-9, K=20, max_steps=200000)
    assert rc == 0
    S = L.LBMSolver(mask, "B", tau, force=(1e-6, 0, 0), precision="fp32", layout="ab",
                    check_interval=20, bounceback="fullway")
    S.step(steps)
    k = S.permeability()[0]
    ko = (tau - 0.5) / 3 * U[0] / 1e-6
    assert abs(k / ko - 1) <= 1e-5


def test_fullway_contract(L, geom, tmp_path):
    mask = geom.sphere_array(12, "sc", r=4.5)
    for layout in ("aa", "sparse"):
        with pytest.raises(L.LBMError):
            L.LBMSolver(mask, "B", 1.0, layout=layout, bounceback="fullway")
    S = L.LBMSolver(mask, "B", 1.0, force=(1e-5, 0, 0), precision="fp64", layout="ab",
                    check_interval=10, bounceback="fullway")
    H = L.LBMSolver(mask, "B", 1.0, precision="fp64", layout="ab")
    assert S.link_counts()[0] == H.link_counts()[0]
    assert np.array_equal(S.link_counts()[1], H.link_counts()[1])
    rc, _ = S.run_to_convergence(1e-10)
    assert rc == 0
    with pytest.raises(L.LBMError):
        S.adjoint(1e-6)
    # a checkpoint keeps the scheme and the bounceback voxels' populations
    path = str(tmp_path / "fw.lbm")
    S.step(7)
    S.save(path)
    R = L.LBMSolver.load(path)
    S.step(25)
    R.step(25)
    assert np.array_equal(S.velocity(), R.velocity())
    S.close()
    H.close()
    R.close()
