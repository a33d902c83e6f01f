"""Bounded domains (Sec. 2.4) on the FP64 oracle: Zou-He density faces in x
and symmetry (mirror) planes in y and z.

Pins:
- a Zou-He face node carries exactly the prescribed density and no
  tangential momentum;
- at steady state the flux through every x-plane is the same (continuity);
- a pressure-driven slit at Lambda = 3/16 has the exact half-link parabola
  as its profile away from the faces (a boundary layer next to each face
  decays exponentially inward), and its k from the pressure drop between
  the face nodes tends to the exact slit value as 1/(Lx - 1) (the Zou-He
  nodes place the prescribed pressure a fixed fraction of a link off the
  node);
- a symmetry plane is the mirror: z planes leave a z-invariant flow equal to
  the periodic one, and a slit of H rows with a wall on one side and a
  symmetry plane on the other is exactly half of a slit of 2H rows, step by
  step.
"""
import numpy as np
import pytest

C19 = np.array([(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
                (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1),
                (1, 0, -1), (-1, 0, 1), (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)])
H, W, TAU, DR = 8, 1, 0.9, 1e-4


def _pressure_slit(ora, geom, Lx, st="E", lam=3 / 16, linear=True, steps=None):
    m = geom.slit(H, W, Lx=Lx, Lz=1)
    S = ora.Solver(m, ora.rates(st, TAU, lam), [0, 0, 0], linear=linear)
    S.set_domain(pressure_x=True, rho_in=1 + DR / 2, rho_out=1 - DR / 2)
    if steps is not None:
        S.step(steps)
        return S, None
    rc, _, U = S.run_to_convergence(1e-12, K=10, max_steps=400000)
    assert rc == 0
    return S, U


def test_zou_he_faces_carry_prescribed_density(ora, geom):
    S, _ = _pressure_slit(ora, geom, 12, steps=37)
    f = S.get_f()[:, 0, :H, :]  # post-collision: mass and momentum of the streamed state
    for x, rho in ((0, 1 + DR / 2), (11, 1 - DR / 2)):
        fx = f[:, :, x]
        assert np.abs(fx.sum(0) - rho).max() <= 1e-14
        for a in (1, 2):
            assert np.abs((fx * C19[:, a, None]).sum(0)).max() <= 1e-16


def test_pressure_driven_flux_is_continuous(ora, geom):
    S, _ = _pressure_slit(ora, geom, 16, st="D", linear=False)
    flux = S.velocity()[0, 0, :, :].sum(0)  # sum over y of u_x, per x
    assert np.ptp(flux) <= 1e-10 * abs(flux.mean())


def test_pressure_driven_slit_is_poiseuille(ora, geom):
    # a boundary layer next to each Zou-He face decays exponentially inward:
    # mid-length of a 48-node slit carries the exact half-link parabola
    k_exact = (H / (H + W)) * (2 * H**2 + 1) / 24
    nu = (TAU - 0.5) / 3
    y = np.arange(1, H + 1) - (H + 1) / 2
    shape = (H / 2) ** 2 - y**2
    dev = {}
    for Lx in (24, 48):
        S, U = _pressure_slit(ora, geom, Lx)
        if Lx == 48:
            u = S.velocity()[0, 0, :H, Lx // 2]
            assert np.abs(u / u.max() - shape / shape.max()).max() <= 1e-10
        k = nu * U[0] / ((DR / 3) / (Lx - 1))
        dev[Lx] = k / k_exact - 1
    assert 0 < dev[24] < 5e-4
    assert abs(dev[24] * 23 / (dev[48] * 47) - 1) < 1e-3


def test_symmetry_z_equals_periodic_for_z_invariant_flow(ora, geom):
    m = geom.slit(H, W, Lx=6, Lz=4)
    u = []
    for sym in (False, True):
        S = ora.Solver(m, ora.rates("D", 1.1), [1e-6, 0, 0])
        if sym:
            S.set_domain(symmetry_z=True)
        S.step(150)
        u.append(S.velocity())
    assert np.abs(u[0] - u[1]).max() <= 1e-15 * np.abs(u[0]).max()


@pytest.mark.parametrize("st,linear", [("B", True), ("C", False)])
def test_symmetry_y_halves_a_slit(ora, geom, st, linear):
    full = geom.slit(2 * H, 1)                 # fluid rows 0..2H-1, wall row 2H
    half = geom.slit(H, 1)                     # fluid rows 0..H-1, wall row H
    Sf = ora.Solver(full, ora.rates(st, 1.0), [1e-5, 0, 0], linear=linear)
    Sh = ora.Solver(half, ora.rates(st, 1.0), [1e-5, 0, 0], linear=linear)
    Sh.set_domain(symmetry_y=True)             # mirror below row 0
    for n in (3, 40, 400):
        Sf.step(n - Sf.steps)
        Sh.step(n - Sh.steps)
        uf = Sf.velocity()[0, 0, :2 * H, 0]
        uh = Sh.velocity()[0, 0, :H, 0]
        assert np.abs(uh - uf[H:]).max() <= 1e-12 * np.abs(uf).max()
        assert np.abs(uh[::-1] - uf[:H]).max() <= 1e-12 * np.abs(uf).max()
