"""The batched sweep against single-lattice runs and the oracle, under both
schedules: the persistent kernel with grid barriers and the stepwise one
(per step, one launch per class of lattices).

Every batch member runs the same per-unit update on the same locations as a
lattice run alone, and the stopping rule is evaluated on the same schedule,
so its step count and populations must be bitwise those of the lone run.
The barrier's bounded wait is exercised by a test hook that makes one block
skip an arrival: the run must end with LBM_ETIMEOUT, not hang.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_11193_gb300 import lbm

    lbm.lib()
    return lbm


def _lattices(geom):
    return [
        dict(mask=geom.sphere_array(16, "sc", c=0.2), set_="B", tau=0.8, force=(1e-5, 0, 0)),
        dict(mask=geom.sphere_array(20, "bcc", c=0.3), set_="D", tau=1.3, force=(1e-5, 0, 0)),
        dict(mask=geom.sphere_array(24, "fcc", c=0.4), set_="E", tau=1.0, Lambda=3 / 8,
             force=(0, 1e-5, 0)),
        dict(mask=geom.boolean((30, 26, 22), 4, 0.45, seed=7)[0], set_="A", tau=0.9,
             force=(1e-5, 0, 0)),
        dict(mask=geom.slit(7, 2, Lx=5, Lz=3), set_="C", tau=1.1, force=(1e-5, 0, 0)),
        dict(mask=geom.random_mask((13, 11, 9), 0.25, seed=3), set_="SRT", tau=0.7,
             force=(1e-5, 2e-6, 0)),
    ]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("layout,npt,rule,solo", [("aa", 1, 0, "auto"), ("sparse", 2, 1, "auto"),
                                                  (None, 0, 1, "auto"), (None, 0, 0, "always")])
def test_batch_bitwise_equals_single_runs(L, geom, precision, layout, npt, rule, solo):
    lats = _lattices(geom)
    B = L.LBMBatch(lats, precision=precision, layout=layout, nodes_per_thread=npt,
                   check_interval=20, max_steps=6000, stop_rule=rule, solo=solo)
    steps, status = B.run(1e-7)
    lay, nps = B.config()
    assert set(lay.tolist()) <= {L.AA, L.SPARSE} and set(nps.tolist()) <= {0, 1, 2}
    if solo == "always":
        assert np.all(nps == 0)  # every lattice ran alone
    elif npt:
        assert np.all(nps == npt)
    if rule == 1:
        assert np.all(status == 0)
    kb = B.permeability()
    for i, l in enumerate(lats):
        S = L.LBMSolver(l["mask"], l["set_"], l["tau"], l.get("Lambda", 3 / 16), l["force"],
                        precision=precision, layout=["ab", "aa", "sparse"][lay[i]],
                        check_interval=20, max_steps=6000, stop_rule=rule)
        rc, st = S.run_to_convergence(1e-7)
        assert rc == status[i] and st == steps[i]
        assert np.array_equal(S.get_populations(), B.lattice(i).get_populations())
        assert np.array_equal(S.converged_permeability(), kb[i], equal_nan=True)


@pytest.mark.parametrize("npt", [1, 2])
@pytest.mark.parametrize("rule", [0, 1])
def test_batch_fp64_matches_oracle(L, ora, geom, rule, npt):
    """Both tile shapes of the persistent kernel (one and two fluid nodes per
    thread) against the oracle's converged permeability."""
    lats = _lattices(geom)[:3]
    B = L.LBMBatch(lats, precision="fp64", layout="sparse", nodes_per_thread=npt,
                   check_interval=10, stop_rule=rule, schedule="persistent")
    steps, status = B.run(1e-9)
    assert np.all(status == 0)
    assert np.all(B.config()[1] == npt)
    kb = B.permeability()
    for i, l in enumerate(lats):
        O = ora.Solver(l["mask"], ora.rates(l["set_"], l["tau"], l.get("Lambda", 3 / 16)),
                       l["force"])
        rc, st, U = O.run_to_convergence(1e-9, K=10, max_steps=100000, rule=rule)
        assert rc == 0 and st == steps[i]
        d = int(np.argmax(np.abs(l["force"])))
        ko = (l["tau"] - 0.5) / 3 * U[d] / l["force"][d]
        assert abs(kb[i][d] - ko) <= 1e-10 * abs(ko)


def test_batch_retires_unstable_and_capped(L, geom):
    lats = _lattices(geom)[:2]
    lats.append(dict(mask=geom.sphere_array(16, "sc", c=0.2), set_="SRT", tau=0.5001,
                     force=(0.5, 0, 0)))
    B = L.LBMBatch(lats, precision="fp32", layout="aa", check_interval=10, max_steps=300,
                   solo="never")
    steps, status = B.run(0.0)  # tol 0: nothing converges
    assert status[2] == -5  # unstable
    assert status[0] == -4 and status[1] == -4 and steps[0] == 300


def test_batch_barrier_timeout_is_reported(L, geom):
    lats = _lattices(geom)
    B = L.LBMBatch(lats, precision="fp32", layout="aa", check_interval=10,
                   barrier_timeout_ms=200, test_skip_block=0, solo="never",
                   schedule="persistent")
    rc = B.run(1e-7, raise_on_failure=False)
    assert rc == -6  # LBM_ETIMEOUT: the waits ran out, the kernel returned
    assert B.run(1e-7, raise_on_failure=False) == -6
    B.close()
    # the device is still usable
    C2 = L.LBMBatch(lats[:2], precision="fp32", layout="aa", check_interval=10, solo="never")
    steps, status = C2.run(1e-7)
    assert np.all(status == 0)


@pytest.mark.parametrize("layout,rule", [("aa", 0), ("sparse", 1), (None, 0), (None, 1)])
def test_batch_stepwise_bitwise_equals_single_runs(L, geom, layout, rule):
    """The stepwise schedule: every chunk launched per step and class; the
    members' step counts, populations and converged k bitwise those of lone
    runs (two collision forms, both parities of the tile lists, ragged
    tiles)."""
    lats = _lattices(geom)
    B = L.LBMBatch(lats, precision="fp32", layout=layout, check_interval=20, max_steps=6000,
                   stop_rule=rule, schedule="stepwise")
    steps, status = B.run(1e-7)
    sw, pe = B.schedule_counts()
    assert sw > 0 and pe == 0
    lay, _ = B.config()
    kb = B.permeability()
    for i, l in enumerate(lats):
        S = L.LBMSolver(l["mask"], l["set_"], l["tau"], l.get("Lambda", 3 / 16), l["force"],
                        precision="fp32", layout=["ab", "aa", "sparse"][lay[i]],
                        check_interval=20, max_steps=6000, stop_rule=rule)
        rc, st = S.run_to_convergence(1e-7)
        assert rc == status[i] and st == steps[i]
        assert np.array_equal(S.get_populations(), B.lattice(i).get_populations())
        assert np.array_equal(S.converged_permeability(), kb[i], equal_nan=True)
        S.close()


def test_batch_schedule_switches_midway(L, geom):
    """Two large lattices (over 10^5 units) run their first chunk with their
    own kernels beside the small ones' persistent launch; without a drive
    they meet the stopping rule at their first check and retire, and the
    small slow ones (tau = 0.6) finish in the persistent kernel alone.  Every
    member still equals its lone run bitwise."""
    big = geom.sphere_array(96, "sc", c=0.1)
    lats = [dict(mask=big, set_="B", tau=1.6, force=(0, 0, 0)),
            dict(mask=big, set_="D", tau=1.6, force=(0, 0, 0))]
    lats += [dict(l, tau=0.6) for l in _lattices(geom)[:3]]
    B = L.LBMBatch(lats, precision="fp32", layout="sparse", check_interval=50, max_steps=20000)
    steps, status = B.run(1e-6)
    sw, pe = B.schedule_counts()
    assert sw > 0 and pe > 0, (sw, pe)
    kb = B.permeability()
    for i, l in enumerate(lats):
        S = L.LBMSolver(l["mask"], l["set_"], l["tau"], l.get("Lambda", 3 / 16), l["force"],
                        precision="fp32", layout="sparse", check_interval=50, max_steps=20000)
        rc, st = S.run_to_convergence(1e-6)
        assert rc == status[i] and st == steps[i]
        assert np.array_equal(S.get_populations(), B.lattice(i).get_populations())
        assert np.array_equal(S.converged_permeability(), kb[i], equal_nan=True)
        S.close()


def test_batch_stepwise_retires_unstable(L, geom):
    lats = _lattices(geom)[:2]
    lats.append(dict(mask=geom.sphere_array(16, "sc", c=0.2), set_="SRT", tau=0.5001,
                     force=(0.5, 0, 0)))
    B = L.LBMBatch(lats, precision="fp32", layout="sparse", check_interval=10, max_steps=300,
                   schedule="stepwise")
    steps, status = B.run(0.0)
    assert status[2] == -5
    assert status[0] == -4 and status[1] == -4 and steps[0] == 300


@pytest.mark.parametrize("rule", [0, 1])
def test_batch_auto_own_kernels_bitwise(L, geom, rule):
    """The automatic schedule: lattices of over 10^5 units (64^3 BCC cells)
    run each chunk with their own graph-replayed kernels, the small ones in
    the persistent launch of the same chunk; every member equals its lone
    run bitwise."""
    m = geom.sphere_array(64, "bcc", c=0.3)
    lats = [dict(mask=m, set_=st, tau=t, Lambda=lam, force=(1e-5, 0, 0))
            for st, t, lam in (("B", 0.8, 3 / 16), ("D", 1.3, 3 / 16), ("C", 0.9, 3 / 16))]
    lats += _lattices(geom)[:3]
    B = L.LBMBatch(lats, precision="fp32", layout="sparse", check_interval=20, max_steps=1200,
                   stop_rule=rule)
    steps, status = B.run(1e-8)
    sw, pe = B.schedule_counts()
    assert sw > 0 and pe > 0, (sw, pe)
    nps = B.config()[1]
    assert np.all(nps[:3] == 0) and np.all(nps[3:] > 0)  # own kernels vs tiles
    kb = B.permeability()
    for i, l in enumerate(lats):
        S = L.LBMSolver(l["mask"], l["set_"], l["tau"], l.get("Lambda", 3 / 16), l["force"],
                        precision="fp32", layout="sparse", check_interval=20, max_steps=1200,
                        stop_rule=rule)
        rc, st = S.run_to_convergence(1e-8)
        assert rc == status[i] and st == steps[i]
        assert np.array_equal(S.get_populations(), B.lattice(i).get_populations())
        assert np.array_equal(S.converged_permeability(), kb[i], equal_nan=True)
        S.close()
