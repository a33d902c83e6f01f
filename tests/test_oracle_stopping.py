"""Stopping rule on voxel media with thin gaps, and the adjoint there.

In gaps one or two voxels wide halfway bounceback reverses almost every
population carrying momentum across the gap, while the collision conserves
momentum, so the step has modes of eigenvalue near -1: the mean velocity
keeps alternating around the fixed point for tens of thousands of steps and
the per-step rule of eq. (convergence) cannot hold.  Rule 1 applies the rule
to the mean of two consecutive steps, which cancels those modes; what it
stops on must be the fixed point, i.e. the two-step mean the iteration keeps
long after.
"""
import numpy as np
import pytest

F = [1e-6, 0.0, 0.0]


@pytest.fixture(scope="module")
def gappy(geom):
    # 32^3 Boolean medium, r = 4, porosity 0.35: contains one-voxel gaps
    return geom.boolean(32, 4, 0.35, seed=1902_11193 + 4)[0]


def test_per_step_rule_stalls_two_step_rule_converges(ora, gappy):
    S = ora.Solver(gappy, ora.rates("D", 1.0), F)
    rc, steps, _ = S.run_to_convergence(1e-6, K=10, max_steps=6000, rule=0)
    assert rc == 1 and steps == 6000  # the per-step change stays ~1e-3
    T = ora.Solver(gappy, ora.rates("D", 1.0), F)
    rc, steps, U = T.run_to_convergence(1e-11, K=10, max_steps=60000, rule=1)
    assert rc == 0
    # long after: consecutive steps still alternate, their mean is what rule 1 stopped on
    T.step(3000)
    a = T.step(1, want_U=True)[0]
    b = T.step(1, want_U=True)[0]
    assert abs(b - a) / abs(b) > 1e-5
    # within the slow modes' remainder (per-step tolerance 1e-11 times a decay
    # time of ~5e3 steps), far inside the +-5e-4 alternation
    assert abs(0.5 * (a + b) - U[0]) <= 1e-6 * abs(U[0])


def test_two_step_rule_equals_per_step_rule_without_gaps(ora, geom):
    """On a sphere array without thin gaps both rules find the same k."""
    mask = geom.sphere_array(12, "bcc", c=0.3)
    S = ora.Solver(mask, ora.rates("B", 0.9), F)
    rc0, _, U0 = S.run_to_convergence(1e-13, K=10, max_steps=100000, rule=0)
    T = ora.Solver(mask, ora.rates("B", 0.9), F)
    rc1, _, U1 = T.run_to_convergence(1e-13, K=10, max_steps=100000, rule=1)
    assert rc0 == 0 and rc1 == 0
    assert abs(U1[0] - U0[0]) <= 1e-10 * abs(U0[0])


def test_adjoint_on_gappy_medium_matches_finite_differences(ora, geom):
    """The averaged adjoint against central differences of the fixed-point k."""
    mask = geom.boolean(24, 3, 0.35, seed=1902_11193 + 6)[0]
    tau, lam, h = 0.9, 3 / 8, 1e-4

    def k_at(t, l, Fv):
        S = ora.Solver(mask, ora.rates("E", t, l), Fv)
        rc, _, U = S.run_to_convergence(1e-13, K=10, max_steps=100000, rule=1)
        assert rc == 0
        return S, (t - 0.5) / 3 * U[0] / Fv[0]

    S, k = k_at(tau, lam, F)
    rc, g, _ = S.adjoint("E", tau, lam, tol=1e-11, max_iter=100000)
    assert rc == 0
    fd_tau = (k_at(tau + h, lam, F)[1] - k_at(tau - h, lam, F)[1]) / (2 * h)
    fd_lam = (k_at(tau, lam + h, F)[1] - k_at(tau, lam - h, F)[1]) / (2 * h)
    assert abs(g["dtau"] * tau / k - fd_tau * tau / k) < 1e-5
    assert abs(g["dLambda"] * lam / k - fd_lam * lam / k) < 1e-5
