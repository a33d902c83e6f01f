"""The paper's own solid boundary (Sec. 3) on the FP64 oracle: the 0/1/2
voxel flags and full-way bounceback.

Full-way bounceback keeps the populations that stream into a bounceback
voxel there for one step and sends them back along the opposite link: the
same reflection as halfway bounceback, one step later.  A steady state has
no time to lose, so the steady flow, and k, are those of halfway bounceback
with the wall at the half-link; the transients differ.  Pins:
- flags against a brute-force classification;
- mass: fluid populations plus the bounceback-voxel populations headed for
  fluid voxels are invariant (streaming permutes them, collisions conserve
  mass, the reflection is a permutation);
- the Poiseuille slit at Lambda = 3/16: the exact half-link parabola;
- a BCC array: converged k equal to the halfway k; after a few steps not.
"""
import numpy as np
import pytest

C19 = np.array([(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
                (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1),
                (1, 0, -1), (-1, 0, 1), (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)])
F = 1e-6


def _brute_flags(mask):
    Lz, Ly, Lx = mask.shape
    out = np.zeros_like(mask)
    for z in range(Lz):
        for y in range(Ly):
            for x in range(Lx):
                if not mask[z, y, x]:
                    continue
                fluid_nb = any(mask[(z + c[2]) % Lz, (y + c[1]) % Ly, (x + c[0]) % Lx] == 0
                               for c in C19[1:])
                out[z, y, x] = 1 if fluid_nb else 2
    return out


@pytest.mark.parametrize("seed,frac", [(1, 0.3), (2, 0.7), (3, 0.9)])
def test_flags_match_brute_force(ora, geom, seed, frac):
    mask = geom.random_mask((7, 6, 5), frac, seed=seed)
    assert np.array_equal(ora.flags(mask), _brute_flags(mask))


def test_flags_of_a_sphere_array(ora, geom):
    mask = geom.sphere_array(12, "sc", r=4.5)
    fl = ora.flags(mask)
    assert np.array_equal(fl, _brute_flags(mask))
    assert (fl == 2).any() and (fl == 1).any()


def _live_mass(f, fl):
    Lz, Ly, Lx = fl.shape
    m = f[:, fl == 0].sum()
    for j in range(1, 19):
        # bounceback-voxel population j heads to x + c_j: counts if that is fluid
        dest = np.roll(fl, shift=(-C19[j][2], -C19[j][1], -C19[j][0]), axis=(0, 1, 2))
        m += f[j][(fl == 1) & (dest == 0)].sum()
    return m


def test_fullway_mass_invariant(ora, geom):
    mask = geom.boolean((14, 12, 10), 3, 0.5, seed=5)[0]
    fl = ora.flags(mask)
    S = ora.Solver(mask, ora.rates("D", 0.8), [1e-4, 2e-5, 0], bounceback="fullway")
    m0 = _live_mass(S.get_f(), fl)
    S.step(300)
    m1 = _live_mass(S.get_f(), fl)
    assert abs(m1 - m0) <= 1e-13 * m0


def test_fullway_slit_is_exact_half_link_parabola(ora, geom):
    H, W, tau, Fx = 8, 2, 0.9, 1e-5
    m = geom.slit(H, W)
    S = ora.Solver(m, ora.rates("E", tau, 3 / 16), [Fx, 0, 0], linear=True, bounceback="fullway")
    rc, _, _ = S.run_to_convergence(1e-15, K=1, max_steps=200000)
    assert rc == 0
    u = S.velocity()[0, 0, :H, 0]
    nu = (tau - 0.5) / 3
    y = np.arange(1, H + 1) - (H + 1) / 2
    exact = Fx / (2 * nu) * ((H / 2) ** 2 - y**2)
    assert np.abs(u - exact).max() <= 1e-9 * exact.max()


def test_fullway_steady_k_equals_halfway(ora, geom):
    mask = geom.sphere_array(10, "bcc", r=3.2)
    ks, early = {}, {}
    for bb in ("halfway", "fullway"):
        S = ora.Solver(mask, ora.rates("D", 1.2), [F, 0, 0], bounceback=bb)
        S.step(8)
        early[bb] = S.mean_velocity()[0]
        rc, _, U = S.run_to_convergence(1e-14, K=10, max_steps=400000)
        assert rc == 0
        ks[bb] = U[0]
    assert abs(ks["fullway"] - ks["halfway"]) <= 1e-9 * abs(ks["halfway"])
    assert abs(early["fullway"] - early["halfway"]) > 1e-3 * abs(early["halfway"])
