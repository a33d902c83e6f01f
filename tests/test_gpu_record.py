"""The record of a stopping-rule run (lbm_convergence_history and the Python
run record) against the oracle stepped by hand.

At every check the library reports the step count, the mean velocity along
the drive that the rule of eq. (convergence) compares and the relative
change.  The oracle, stepped chunk by chunk with the velocity measured in
the same steps, gives the same sequence: the FP64 path within 1e-11 of each
value (the velocity's parity bound), the steps exactly.
"""
import json

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

F = (1e-4, 0.0, 0.0)


@pytest.fixture(scope="module")
def L():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_11193_gb300 import lbm

    lbm.lib()
    return lbm


def _oracle_history(ora, mask, st, tau, K, rule, n_checks):
    """The oracle's checks: (step, U_b, |U_b - U_a| / |U_b|) per chunk of K
    steps; rule 0 compares the chunk's last two steps, rule 1 the means of
    its last three steps taken two at a time."""
    O = ora.Solver(mask, ora.rates(st, tau), F)
    out, done = [], 0
    for _ in range(n_checks):
        if rule == 0:
            O.step(K - 2)
            Ua = O.step(1, want_U=True)[0]
            Ub = O.step(1, want_U=True)[0]
        else:
            O.step(K - 3)
            U1 = O.step(1, want_U=True)[0]
            U2 = O.step(1, want_U=True)[0]
            U3 = O.step(1, want_U=True)[0]
            Ua, Ub = 0.5 * (U1 + U2), 0.5 * (U2 + U3)
        done += K
        out.append((done, Ub, abs(Ub - Ua) / abs(Ub)))
    return out


@pytest.mark.parametrize("layout", ["aa", "sparse"])
@pytest.mark.parametrize("rule", [0, 1])
def test_history_matches_oracle(L, ora, geom, layout, rule):
    mask = geom.sphere_array(16, "bcc", c=0.3)
    K, tol = 20, 1e-6
    S = L.LBMSolver(mask, "B", 0.9, force=F, precision="fp64", layout=layout, check_interval=K,
                    stop_rule=rule, max_steps=20000)
    rc, steps = S.run_to_convergence(tol)
    assert rc == 0
    h = S.convergence_history()
    assert len(h) == steps // K and h["step"][-1] == steps
    assert np.all(np.diff(h["step"]) == K)
    assert h["change"][-1] <= tol and np.all(h["change"][:-1] > tol)
    assert h["U"][-1] == S.converged_velocity()[0]
    ref = _oracle_history(ora, mask, "B", 0.9, K, rule, len(h))
    for (st, U, ch), r in zip(ref, h):
        assert r["step"] == st
        assert abs(r["U"] - U) <= 1e-11 * abs(U)
        # the change is a difference of nearby values: compare it absolutely
        assert abs(r["change"] - ch) <= 1e-9
    S.close()


def test_run_record_is_json(L, geom):
    mask = geom.sphere_array(16, "sc", c=0.2)
    S = L.LBMSolver(mask, "D", 1.0, force=F, precision="fp32", layout="sparse",
                    check_interval=50, max_steps=50000)
    rc, steps = S.run_to_convergence(1e-6)
    assert rc == 0
    rec = json.loads(json.dumps(S.run_record()))
    assert rec["run"]["status"] == "OK" and rec["run"]["steps"] == steps
    assert rec["precision"] == "fp32" and rec["layout"] == "sparse"
    assert rec["dims"] == [16, 16, 16] and rec["steps_total"] == steps
    assert len(rec["history"]) == steps // 50
    assert rec["history"][-1]["change"] <= 1e-6
    assert rec["k_conv"][0] == S.converged_permeability()[0]
    # a second run starts a new history
    S.run_to_convergence(1e-6)
    assert len(S.convergence_history()) == 1
    S.close()
