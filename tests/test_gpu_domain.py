"""Bounded domains (Sec. 2.4) on the CUDA path: Zou-He density faces in x,
symmetry planes in y and z, and the paper's 5-layer inlet/outlet padding.

The AB bounded kernel against the FP64 oracle's bounded solver at equal
step counts (velocity field), converged permeability from the pressure
gradient in FP64 and FP32, and the option's contract.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

DR = 1e-4


@pytest.fixture(scope="module")
def L():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_11193_gb300 import lbm

    lbm.lib()
    return lbm


def _cases(geom):
    sample = geom.boolean((16, 14, 12), 3, 0.55, seed=1902_11193 + 9)[0]
    return {
        # pressure-driven slit, walls in y, mirror planes in z
        "slit": (geom.slit(8, 1, Lx=16, Lz=3), dict(pressure=True, sym="z"), (0, 0, 0)),
        # a padded Boolean sample, pressure-driven, mirror planes in y and z
        "padded": (geom.pad_x(sample, 5), dict(pressure=True, sym="yz"), (0, 0, 0)),
        # body force along x (periodic), mirror planes in y only
        "mirror_y": (geom.sphere_array(12, "bcc", c=0.3), dict(pressure=False, sym="y"),
                     (1e-5, 2e-6, 0)),
    }


def _oracle(ora, mask, st, tau, kind, F):
    O = ora.Solver(mask, ora.rates(st, tau), list(F))
    O.set_domain(pressure_x=kind["pressure"], rho_in=1 + DR / 2, rho_out=1 - DR / 2,
                 symmetry_y="y" in kind["sym"], symmetry_z="z" in kind["sym"])
    return O


def _gpu(L, mask, st, tau, kind, F, precision, **kw):
    return L.LBMSolver(mask, st, tau, force=F, precision=precision, layout="ab",
                       pressure=(1 + DR / 2, 1 - DR / 2) if kind["pressure"] else None,
                       symmetry=kind["sym"], **kw)


@pytest.mark.parametrize("name", ["slit", "padded", "mirror_y"])
def test_bounded_fp64_matches_oracle(L, ora, geom, name):
    mask, kind, F = _cases(geom)[name]
    O = _oracle(ora, mask, "D", 0.9, kind, F)
    S = _gpu(L, mask, "D", 0.9, kind, F, "fp64")
    for n in (1, 9, 60):
        O.step(n - O.steps)
        S.step(n - S.steps)
        # the oracle carries unshifted populations near 1/3: its roundings are
        # ~1e-13 of the density and velocity deviations per operation (the
        # FP64 stress-test bar, 1e-11 relative), and at a Zou-He face it forms
        # j_x = rho - S_0 - 2 S_out from terms near 1, ~1e-16 absolute per
        # face node and step; over 60 steps a 5e-15 absolute floor
        uo, ug = O.velocity(), S.velocity()
        assert np.abs(ug - uo).max() <= 1e-11 * np.abs(uo).max() + 5e-15
        Uo = O.mean_velocity()
        assert np.abs(S.mean_velocity() - Uo).max() <= 1e-11 * np.abs(Uo).max() + 5e-15
    S.close()


@pytest.mark.parametrize("precision,bar", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_pressure_driven_permeability(L, ora, geom, precision, bar):
    mask, kind, F = _cases(geom)["padded"]
    st, tau = "B", 1.0
    O = _oracle(ora, mask, st, tau, kind, F)
    rc, steps, U = O.run_to_convergence(1e-10, K=20, max_steps=200000)
    assert rc == 0
    Lx = mask.shape[2]
    k_ora = (tau - 0.5) / 3 * U[0] * (Lx - 1) / (DR / 3)
    S = _gpu(L, mask, st, tau, kind, F, precision, check_interval=20)
    S.step(steps)
    k = S.permeability()
    assert np.isnan(k[1]) and np.isnan(k[2])
    assert abs(k[0] / k_ora - 1) <= bar
    S.close()


def test_bounded_contract(L, geom, tmp_path):
    mask, kind, F = _cases(geom)["padded"]
    for kw in (dict(layout="aa"), dict(layout="sparse"), dict(layout="ab", bounceback="fullway")):
        with pytest.raises(L.LBMError):
            L.LBMSolver(mask, "B", 1.0, force=(0, 0, 0), pressure=(1.0001, 0.9999), **kw)
    with pytest.raises(L.LBMError):  # a pressure drive takes no body force
        L.LBMSolver(mask, "B", 1.0, force=(1e-6, 0, 0), layout="ab", pressure=(1.0001, 0.9999))
    with pytest.raises(L.LBMError):  # inlet and outlet need distinct planes
        L.LBMSolver(mask[:, :, :1], "B", 1.0, force=(0, 0, 0), layout="ab",
                    pressure=(1.0001, 0.9999))
    S = _gpu(L, mask, "B", 1.0, kind, F, "fp64", check_interval=20)
    rc, _ = S.run_to_convergence(1e-8)
    assert rc == 0
    with pytest.raises(L.LBMError):
        S.adjoint(1e-6)
    path = str(tmp_path / "bounded.lbm")
    S.save(path)
    R = L.LBMSolver.load(path)
    S.step(30)
    R.step(30)
    assert np.array_equal(S.velocity(), R.velocity())
    assert np.array_equal(S.permeability(), R.permeability(), equal_nan=True)
    S.close()
    R.close()
