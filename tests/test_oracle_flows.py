"""Flow-level pins of the FP64 oracle: analytic Stokes solutions and the
paper's central claim.

(a) Poiseuille flow in a periodic slit: with halfway bounceback and Lambda =
    3/16 the wall sits exactly at the half-link for any tau (Sec. 2.3, Set E
    discussion); other Lambda values shift it by a slip that is uniform,
    tau- and width-independent and linear in Lambda.
(a) Square duct: the continuum series solution (textbook Fourier series for
    a rectangular duct), approached at second order in the resolution.
(b) Dilute simple-cubic sphere arrays: Hasimoto's drag expansion.
(c)-(e) live in test_oracle_pins.py.
Paper's claim (Secs. 4.1-4.3): Sets B, D and E give tau-independent
permeability for Stokes flow; SRT, A and C do not.
"""
import numpy as np
import pytest

F = 1e-6


def _slit_profile(ora, geom, H, W, tau, lam, linear=True, Fx=1e-5):
    m = geom.slit(H, W)
    S = ora.Solver(m, ora.rates("E", tau, lam), [Fx, 0, 0], linear=linear)
    rc, steps, _ = S.run_to_convergence(1e-15, K=1, max_steps=200000)
    assert rc == 0
    u = S.velocity()[0, 0, :H, 0]
    nu = (tau - 0.5) / 3
    y = np.arange(1, H + 1) - (H + 1) / 2
    exact = Fx / (2 * nu) * ((H / 2) ** 2 - y**2)
    return S, u, exact, nu


@pytest.mark.parametrize("H,W,tau", [(4, 1, 1.0), (7, 2, 0.6), (10, 1, 1.7)])
@pytest.mark.parametrize("linear", [True, False])
def test_poiseuille_slit_exact_at_magic_3_16(ora, geom, H, W, tau, linear):
    S, u, exact, nu = _slit_profile(ora, geom, H, W, tau, 3 / 16, linear)
    assert np.abs(u - exact).max() <= 1e-12 * exact.max() * 10
    k = S.permeability(tau)[0]
    k_exact = H * (2 * H * H + 1) / (24 * (H + W))  # node sum of the parabola
    assert abs(k - k_exact) <= 1e-11 * k_exact


def test_slit_slip_linear_in_lambda(ora, geom):
    slips = {}
    for lam in (1 / 64, 1 / 4, 3 / 8):
        vals = []
        for H, W, tau in ((4, 1, 1.0), (7, 2, 0.6), (10, 1, 1.7)):
            _, u, exact, nu = _slit_profile(ora, geom, H, W, tau, lam, Fx=1e-5)
            d = (u - exact) * nu / 1e-5
            assert np.ptp(d) < 1e-9  # uniform across the channel
            vals.append(d.mean())
        assert np.ptp(vals) < 1e-9  # independent of width and tau
        slips[lam] = np.mean(vals)
    lams = np.array(sorted(slips))
    d = np.array([slips[x] for x in lams])
    slope, icept = np.polyfit(lams, d, 1)
    assert np.abs(slope * lams + icept - d).max() < 1e-9  # collinear
    assert abs(slope * 3 / 16 + icept) < 1e-9  # vanishes at Lambda = 3/16


def _duct_C():
    n = np.arange(1, 2001, 2)
    return (1 - 192 / np.pi**5 * np.sum(np.tanh(n * np.pi / 2) / n**5)) / 12


def test_duct_converges_second_order(ora, geom):
    C = _duct_C()
    assert abs(C - 0.0351442537) < 1e-9
    errs = []
    for a in (8, 16, 32):
        S = ora.Solver(geom.duct(a), ora.rates("B", 1.6), [F, 0, 0], linear=True)
        rc, _, U = S.run_to_convergence(1e-13, K=10, max_steps=400000)
        assert rc == 0
        k = (1.6 - 0.5) / 3 * U[0] / F
        errs.append(k / (C * a**4 / (a + 1) ** 2) - 1)
    assert abs(errs[0]) < 0.02
    for e0, e1 in zip(errs, errs[1:]):
        assert 3.0 < e0 / e1 < 5.0


def test_duct_tau_independent(ora, geom):
    ks = []
    for tau in (0.7, 1.0, 1.6):
        S = ora.Solver(geom.duct(8), ora.rates("B", tau), [F, 0, 0], linear=True)
        rc, _, U = S.run_to_convergence(1e-15, K=10, max_steps=400000)
        assert rc == 0
        ks.append((tau - 0.5) / 3 * U[0] / F)
    assert np.ptp(ks) / np.mean(ks) < 1e-10


def _k_bcc(ora, geom, st, tau, lam):
    m = geom.sphere_array(10, "bcc", r=3.2)
    S = ora.Solver(m, ora.rates(st, tau, lam), [F, 0, 0], linear=True)
    rc, _, U = S.run_to_convergence(1e-15, K=10, max_steps=400000)
    assert rc == 0
    return (tau - 0.5) / 3 * U[0] / F


@pytest.mark.parametrize("st,lam", [("B", 3 / 16), ("D", 3 / 16), ("E", 1 / 64), ("E", 3 / 8)])
def test_tau_independent_sets(ora, geom, st, lam):
    ks = [_k_bcc(ora, geom, st, tau, lam) for tau in (0.6, 1.0, 2.0)]
    assert np.ptp(ks) / np.mean(ks) < 1e-10


@pytest.mark.parametrize("st", ["SRT", "A", "C"])
def test_tau_dependent_sets(ora, geom, st):
    ks = [_k_bcc(ora, geom, st, tau, 3 / 16) for tau in (0.6, 1.0, 2.0)]
    assert np.ptp(ks) / np.mean(ks) > 0.05
    if st == "SRT":
        assert ks[0] < ks[1] < ks[2]  # SRT permeability grows with tau (Sec. 4.3)


def _hasimoto_K(c):
    """Hasimoto (1959) drag factor of a simple-cubic array, leading terms:
    K = 1 / (1 - 1.7601 c^(1/3) + c - 1.5593 c^2)."""
    return 1.0 / (1 - 1.7601 * c ** (1 / 3) + c - 1.5593 * c**2)


@pytest.mark.parametrize("r", [5, 6])
def test_hasimoto_dilute_sc_array(ora, geom, r):
    L = 32
    m = geom.sphere_array(L, "sc", r=r)
    ns = int(m.sum())
    a = (3 * ns / (4 * np.pi)) ** (1 / 3)  # volume-equivalent radius of the voxel sphere
    c = ns / m.size
    tau = 2.5  # Set B: k does not depend on tau, a large tau converges fastest
    S = ora.Solver(m, ora.rates("B", tau), [F, 0, 0], linear=True)
    rc, _, U = S.run_to_convergence(1e-8, K=10, max_steps=400000)
    assert rc == 0
    k = (tau - 0.5) / 3 * U[0] / F
    k_h = L**3 / (6 * np.pi * a * _hasimoto_K(c))
    assert abs(k / k_h - 1) < 0.02
