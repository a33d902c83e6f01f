"""Pins of the oracle's steady fixed-point adjoint.

The gradient of a converged permeability is defined by finite differences of
that permeability: each adjoint gradient is checked against central
differences (step 1e-4, FP64 forward solves converged to a per-step change of
1e-15).  The transposition itself is checked by the dot-product identity
<L v, w> = <v, L^T w>, with L v taken as a central difference of the forward
step (exact for the quadratic collision up to rounding).  Linear Stokes
(quadratic terms dropped) with the TRT-like sets makes k independent of tau
and of |F|, so those gradients vanish.
"""
import numpy as np
import pytest

F = [1e-5, 0.0, 0.0]
H = 1e-4


@pytest.fixture(scope="module")
def cell(geom):
    return geom.sphere_array(10, "bcc", r=3.2)


def _k(ora, mask, s, F_, tau, linear):
    S = ora.Solver(mask, s, F_, linear=linear)
    rc, _, U = S.run_to_convergence(1e-15, K=10, max_steps=400000)
    assert rc == 0
    return S, (tau - 0.5) / 3 * U[0] / F_[0]


def _rates(ora, st, tau, lam=None, Lq=None, Lm=None):
    if Lq is not None:
        return ora.rates_magic(tau, Lq, Lm)
    return ora.rates(st, tau, lam if lam is not None else 3 / 16)


@pytest.mark.parametrize("st,lam", [("E", 3 / 8), ("D", None), ("A", None), ("SRT", None)])
def test_adjoint_matches_finite_differences(ora, cell, st, lam):
    tau = 0.9
    S, k = _k(ora, cell, _rates(ora, st, tau, lam), F, tau, False)
    rc, g, _ = S.adjoint(st, tau, lam or 3 / 16, tol=1e-12)
    assert rc == 0

    def fd(rp, rm, Fp=F, Fm=F, taup=tau, taum=tau):
        return _k(ora, cell, rp, Fp, taup, False)[1], _k(ora, cell, rm, Fm, taum, False)[1]

    kp, km = fd(_rates(ora, st, tau + H, lam), _rates(ora, st, tau - H, lam), taup=tau + H,
                taum=tau - H)
    assert abs(g["dtau"] * tau / k - (kp - km) / (2 * H) * tau / k) < 1e-6
    s0 = _rates(ora, st, tau, lam)
    kp, km = fd(s0, s0, [F[0] * (1 + H), 0, 0], [F[0] * (1 - H), 0, 0])
    assert abs(g["dFx"] * F[0] / k - (kp - km) / (2 * H)) < 1e-6 * k / k
    if st == "E":
        kp, km = fd(_rates(ora, st, tau, lam + H), _rates(ora, st, tau, lam - H))
        assert abs(g["dLambda"] * lam / k - (kp - km) / (2 * H) * lam / k) < 1e-6
    if st == "D":
        kp, km = fd(_rates(ora, st, tau, Lq=3 / 16 + H, Lm=3 / 8),
                    _rates(ora, st, tau, Lq=3 / 16 - H, Lm=3 / 8))
        assert abs(g["dLambda_q"] * (3 / 16) / k - (kp - km) / (2 * H) * (3 / 16) / k) < 1e-6
        kp, km = fd(_rates(ora, st, tau, Lq=3 / 16, Lm=3 / 8 + H),
                    _rates(ora, st, tau, Lq=3 / 16, Lm=3 / 8 - H))
        assert abs(g["dLambda_m"] * (3 / 8) / k - (kp - km) / (2 * H) * (3 / 8) / k) < 1e-6
    if st in ("A", "SRT"):
        assert np.isnan(g["dLambda"]) and np.isnan(g["dLambda_q"])


@pytest.mark.parametrize("st,lam", [("B", 3 / 16), ("D", 3 / 16), ("E", 1 / 64)])
def test_adjoint_linear_stokes_tau_and_force_independent(ora, cell, st, lam):
    tau = 1.3
    S, k = _k(ora, cell, _rates(ora, st, tau, lam), F, tau, True)
    rc, g, _ = S.adjoint(st, tau, lam, tol=1e-13)
    assert rc == 0
    # dk/dtau is the cancellation of dJ/dtau = U/(3F) and the collision term,
    # both O(k/nu) and each accurate to ~1e-8 (the rate formulas are
    # differenced in tau with step 1e-5); the tau-dependent sets give 0.16-0.68
    assert abs(g["dtau"] * tau / k) < 1e-7
    assert abs(g["dFx"] * F[0] / k) < 1e-8
    assert abs(g["dFy"]) < 1e-6 * abs(k / F[0]) and abs(g["dFz"]) < 1e-6 * abs(k / F[0])


def test_adjoint_step_is_the_transpose(ora, geom):
    """<L v, w> = <v, L^T w> for the linearised step h -> S C(h)."""
    mask = geom.random_mask((6, 5, 4), 0.3, seed=8)
    s = ora.rates("D", 0.8)
    Fv = [2e-3, -1e-3, 5e-4]
    S = ora.Solver(mask, s, Fv)
    rng = np.random.default_rng(4)
    _, w_, _ = ora.lattice()
    fluid = (mask == 0)[None]
    f0 = S.get_f() * (1 + 0.05 * rng.standard_normal((19,) + mask.shape))
    f0 = np.where(fluid, f0, S.get_f())
    S.set_f(f0)
    h0 = S.stream_field(f0)
    v = rng.standard_normal((19,) + mask.shape) * fluid
    w = rng.standard_normal((19,) + mask.shape) * fluid
    eps = 1e-3

    def forward(hv):
        T = ora.Solver(mask, s, Fv)
        T.set_f(T.unstream_field(hv))
        T.step(1)
        return T.stream_field(T.get_f())

    Lv = (forward(h0 + eps * v) - forward(h0 - eps * v)) / (2 * eps)
    LTw = S.adjoint_apply(w)
    lhs, rhs = np.sum(Lv * w * fluid), np.sum(v * LTw)
    assert abs(lhs - rhs) <= 1e-11 * max(abs(lhs), 1.0)


def _k_after(ora, mask, s, F, tau, n):
    S = ora.Solver(mask, s, F)
    S.step(n)
    return (tau - 0.5) / 3 * S.mean_velocity()[0] / F[0]


def test_transient_adjoint_matches_central_differences(ora, geom):
    """The gradient of k after n steps from rest (reverse accumulation through
    every step) against central differences of the oracle's own k(n)."""
    mask = geom.sphere_array(8, "bcc", r=2.4)
    tau, n, F = 0.9, 25, [1e-5, 2e-6, 0.0]
    S = ora.Solver(mask, ora.rates("D", tau), F)
    rc, g = S.adjoint_transient("D", tau, n=n)
    assert rc == 0 and S.steps == n
    k0 = _k_after(ora, mask, ora.rates("D", tau), F, tau, n)
    h = 1e-4
    fd = {
        "dtau": (_k_after(ora, mask, ora.rates("D", tau + h), F, tau + h, n)
                 - _k_after(ora, mask, ora.rates("D", tau - h), F, tau - h, n)) / (2 * h),
        "dLambda_q": (_k_after(ora, mask, ora.rates_magic(tau, 3 / 16 + h, 3 / 8), F, tau, n)
                      - _k_after(ora, mask, ora.rates_magic(tau, 3 / 16 - h, 3 / 8), F, tau, n)) / (2 * h),
        "dLambda_m": (_k_after(ora, mask, ora.rates_magic(tau, 3 / 16, 3 / 8 + h), F, tau, n)
                      - _k_after(ora, mask, ora.rates_magic(tau, 3 / 16, 3 / 8 - h), F, tau, n)) / (2 * h),
    }
    dF = 1e-4 * F[0]
    fd["dFx"] = (_k_after(ora, mask, ora.rates("D", tau), [F[0] + dF, F[1], 0], tau, n)
                 - _k_after(ora, mask, ora.rates("D", tau), [F[0] - dF, F[1], 0], tau, n)) / (2 * dF)
    scale = {"dtau": tau, "dLambda_q": 3 / 16, "dLambda_m": 3 / 8, "dFx": F[0]}
    for key, want in fd.items():
        assert abs(g[key] - want) * scale[key] <= 1e-7 * abs(k0), key


def test_transient_adjoint_tends_to_steady(ora, geom):
    """Once k(n) has stopped changing, the transient gradient is the steady
    adjoint's."""
    mask = geom.sphere_array(6, "bcc", r=1.8)
    tau, F = 1.4, [1e-5, 0.0, 0.0]
    A = ora.Solver(mask, ora.rates("B", tau), F)
    rc, g_tr = A.adjoint_transient("B", tau, n=500)
    assert rc == 0
    B = ora.Solver(mask, ora.rates("B", tau), F)
    rc, _, _ = B.run_to_convergence(1e-15, K=10, max_steps=100000)
    assert rc == 0
    rc, g_st, _ = B.adjoint("B", tau, tol=1e-14)
    assert rc == 0
    k = A.permeability(tau)[0]
    for key, sc in (("dtau", tau), ("dLambda", 3 / 16), ("dFx", F[0])):
        assert abs(g_tr[key] - g_st[key]) * sc <= 1e-8 * abs(k), key
