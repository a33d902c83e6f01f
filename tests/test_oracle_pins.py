"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each check is computed here independently of the oracle's own code path:
textbook lattice identities, the paper's equilibrium written out as an
explicit population formula (eq. BGK-EDF) and projected with numpy, the Guo
forcing moments derived by hand, the Table 2 closed forms evaluated by hand,
and a separately written BGK+Guo collision (Sec. 2.2.2: all rates 1/tau is
SRT).
"""
import numpy as np
import pytest

from conftest import golden


def _c(ora):
    c, w, opp = ora.lattice()
    return c.astype(float), w, opp


def test_lattice_isotropy(ora):
    c, w, opp = _c(ora)
    assert np.isclose(w.sum(), 1.0, atol=1e-15)
    assert np.allclose(w @ c, 0.0, atol=1e-15)
    # second-order isotropy: sum w c_a c_b = c_s^2 delta_ab, c_s^2 = 1/3
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), np.eye(3) / 3, atol=1e-15)
    # fourth-order isotropy: sum w c_a c_b c_c c_d = c_s^4 (d_ab d_cd + d_ac d_bd + d_ad d_bc)
    T = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    d = np.eye(3)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9
    assert np.allclose(T, iso, atol=1e-15)
    for i in range(19):
        assert np.array_equal(c[opp[i]], -c[i])
    assert len({tuple(v) for v in c}) == 19


def test_moment_matrix_orthogonal_norms(ora):
    M = ora.moment_matrix()
    D = M @ M.T
    off = D - np.diag(np.diag(D))
    assert np.abs(off).max() == 0.0
    want = np.array([float(r[1]) for r in golden("moment_norms.txt")])
    assert np.array_equal(np.diag(D), want)
    # momentum rows are the velocity components: m_{3,5,7} = j (Sec. 2.2.1)
    c, w, _ = _c(ora)
    assert np.array_equal(M[3], c[:, 0]) and np.array_equal(M[5], c[:, 1])
    assert np.array_equal(M[7], c[:, 2]) and np.array_equal(M[0], np.ones(19))


def test_rest_state_moments(ora):
    M = ora.moment_matrix()
    _, w, _ = _c(ora)
    want = np.array([float(r[1]) for r in golden("rest_moments.txt")])
    assert np.allclose(M @ w, want, atol=1e-14)
    assert np.allclose(ora.meq(1.0, [0, 0, 0]), want, atol=0)


def _feq_incompressible(c, w, rho, j, linear=False):
    """eq. (BGK-EDF) in the incompressible form that matches the 1/rho0
    moments of eq. (MRT Equi): f_i = w_i [rho + 3 c.j + 9/2 (c.j)^2 - 3/2 j.j]."""
    cj = c @ j
    q = 0.0 if linear else 1.0
    return w * (rho + 3 * cj + q * (4.5 * cj**2 - 1.5 * (j @ j)))


@pytest.mark.parametrize("linear", [False, True])
def test_meq_is_projection_of_bgk_equilibrium(ora, linear):
    c, w, _ = _c(ora)
    M = ora.moment_matrix()
    rng = np.random.default_rng(7)
    for _ in range(20):
        rho = 1 + 0.1 * rng.standard_normal()
        j = 0.05 * rng.standard_normal(3)
        want = M @ _feq_incompressible(c, w, rho, j, linear)
        got = ora.meq(rho, j, linear)
        assert np.allclose(got, want, rtol=0, atol=1e-14), (got - want)


def test_guo_populations_moments(ora):
    """Guo forcing (eq. Guo_Forcing) carries zero mass, momentum F and second
    moment u F + F u: the properties that define it."""
    c, w, _ = _c(ora)
    rng = np.random.default_rng(11)
    for _ in range(10):
        u = 0.05 * rng.standard_normal(3)
        F = 1e-3 * rng.standard_normal(3)
        Fi = ora.guo_populations(u, F)
        assert abs(Fi.sum()) < 1e-17
        assert np.allclose(Fi @ c, F, atol=1e-17)
        assert np.allclose(np.einsum("i,ia,ib->ab", Fi, c, c),
                           np.outer(u, F) + np.outer(F, u), atol=1e-17)
        Fl = ora.guo_populations(u, F, linear=True)
        assert np.allclose(Fl, 3 * w * (c @ F), atol=1e-18)


def _mF_closed_form(u, F):
    """Moments of the Guo term derived by hand (u = j / rho0)."""
    ux, uy, uz = u
    Fx, Fy, Fz = F
    uF = u @ F
    m = np.zeros(19)
    m[1] = 38 * uF
    m[2] = -11 * uF
    m[3], m[5], m[7] = Fx, Fy, Fz
    m[4], m[6], m[8] = -2 / 3 * Fx, -2 / 3 * Fy, -2 / 3 * Fz
    m[9] = 2 * (2 * ux * Fx - uy * Fy - uz * Fz)
    m[10] = -0.5 * m[9]
    m[11] = 2 * (uy * Fy - uz * Fz)
    m[12] = -0.5 * m[11]
    m[13] = ux * Fy + uy * Fx
    m[14] = uy * Fz + uz * Fy
    m[15] = ux * Fz + uz * Fx
    return m


def test_force_moments_closed_form(ora):
    rng = np.random.default_rng(3)
    for _ in range(20):
        u = 0.05 * rng.standard_normal(3)
        F = 1e-3 * rng.standard_normal(3)
        got = ora.force_moments(u, F)
        want = _mF_closed_form(u, F)
        assert np.abs(got - want).max() <= 1e-15 * np.abs(F).max() * 10
        lin = ora.force_moments(u, F, linear=True)
        assert np.abs(lin - _mF_closed_form(np.zeros(3), F)).max() <= 1e-17


def test_rates_table2(ora):
    for st, tau, lam, k, val in golden("rates_table2.txt"):
        s = ora.rates(st, float(tau), float(lam) if float(lam) > 0 else 3 / 16)
        assert abs(s[int(k)] - float(val)) < 1e-14, (st, tau, lam, k, s[int(k)])


@pytest.mark.parametrize("tau", [0.55, 0.6, 0.8, 1.0, 1.15, 1.3, 1.6, 2.0, 3.0])
def test_rates_structure_and_magic(ora, tau):
    sn = 1 / tau
    odd = [4, 6, 8, 16, 17, 18]
    even = [1, 2, 9, 10, 11, 12, 13, 14, 15]
    magic = lambda sp, sm: (1 / sp - 0.5) * (1 / sm - 0.5)  # eq. (Magic param)
    for st in ("A", "B", "C", "D", "E", "SRT"):
        s = ora.rates(st, tau, 0.3)
        assert s[0] == s[3] == s[5] == s[7] == 0.0
        assert all(s[k] == sn for k in (9, 11, 13, 14, 15))
        assert all(0 < s[k] < 2 for k in odd + even)
    sB = ora.rates("B", tau)
    assert all(sB[k] == sn for k in even)
    assert all(abs(magic(sn, sB[k]) - 3 / 16) < 1e-14 for k in odd)
    sD = ora.rates("D", tau)
    assert all(abs(magic(sn, sD[k]) - 3 / 16) < 1e-14 for k in (4, 6, 8))
    assert all(abs(magic(sn, sD[k]) - 3 / 8) < 1e-14 for k in (16, 17, 18))
    sA = ora.rates("A", tau)
    assert all(abs(magic(sn, sA[k]) - 3 / 16) < 1e-14 for k in odd)
    for lam in (1 / 64, 1 / 8, 3 / 16, 1 / 4, 3 / 8, 1.0):
        sE = ora.rates("E", tau, lam)
        assert all(sE[k] == sn for k in even)
        assert all(abs(magic(sn, sE[k]) - lam) < 1e-14 for k in odd)
    # Set B is Set E at Lambda = 3/16 (Sec. 2.3)
    assert np.allclose(ora.rates("E", tau, 3 / 16), sB, rtol=0, atol=1e-15)
    # Set E at Lambda = (tau - 1/2)^2 gives every rate 1/tau, i.e. SRT
    sE = ora.rates("E", tau, (tau - 0.5) ** 2)
    assert np.allclose(sE[even + odd], sn, atol=1e-14)


def test_rates_reject_bad_tau(ora):
    with pytest.raises(ValueError):
        ora.rates("B", 0.5)
    with pytest.raises(ValueError):
        ora.rates("E", 1.0, 0.0)


def _bgk_guo_step(c, w, f, tau, F, linear=False):
    """BGK with Guo forcing, written independently: f* = f - (f - f^eq)/tau
    + (1 - 1/(2 tau)) F_i, shifted momentum j = sum c f + F/2, rho0 = 1."""
    rho = f.sum()
    j = f @ c + 0.5 * F
    feq = _feq_incompressible(c, w, rho, j, linear)
    u = np.zeros(3) if linear else j
    Fi = w * (3 * ((c - u) @ F) + 9 * (c @ u) * (c @ F))
    return f - (f - feq) / tau + (1 - 0.5 / tau) * Fi


@pytest.mark.parametrize("tau", [0.6, 1.0, 1.7])
@pytest.mark.parametrize("linear", [False, True])
def test_mrt_reduces_to_bgk(ora, tau, linear):
    c, w, _ = _c(ora)
    rng = np.random.default_rng(5)
    F = np.array([1e-3, -2e-4, 5e-4])
    for s in (ora.rates("SRT", tau), ora.rates("E", tau, (tau - 0.5) ** 2)):
        for _ in range(10):
            f = w * (1 + 0.05 * rng.standard_normal(19))
            got = ora.collide(f, s, F, linear)
            want = _bgk_guo_step(c, w, f, tau, F, linear)
            assert np.abs(got - want).max() <= 1e-14


def test_collision_conserves_mass_and_adds_force(ora):
    c, w, _ = _c(ora)
    rng = np.random.default_rng(9)
    F = np.array([2e-4, 1e-4, -3e-4])
    for st in ("A", "B", "C", "D", "E"):
        s = ora.rates(st, 0.9, 3 / 8)
        f = w * (1 + 0.05 * rng.standard_normal(19))
        fo = ora.collide(f, s, F)
        assert abs(fo.sum() - f.sum()) < 4e-16 * 19
        # momentum gains the full force per step: sum c f* = sum c f + F
        assert np.allclose(fo @ c, f @ c + F, atol=1e-16)


def test_rest_state_fixed_point(ora, geom):
    mask = geom.random_mask((6, 5, 4), 0.3, seed=2)
    for st in ("A", "C", "D"):
        S = ora.Solver(mask, ora.rates(st, 0.8), [0, 0, 0])
        f0 = S.get_f()
        S.step(50)
        assert np.abs(S.get_f() - f0).max() <= 1e-15


def test_mass_conservation(ora, geom):
    mask = geom.random_mask((7, 6, 5), 0.35, seed=4)
    c, w, _ = _c(ora)
    S = ora.Solver(mask, ora.rates("C", 0.7), [1e-4, 2e-5, 0.0])
    rng = np.random.default_rng(1)
    f = S.get_f()
    f = f * (1 + 0.02 * rng.standard_normal(f.shape))
    f[:, mask == 1] = 0.0
    S.set_f(f)
    m0 = f.sum()
    S.step(500)
    m1 = S.get_f().sum()
    assert abs(m1 - m0) / m0 <= 1e-13


def _brute_links(mask):
    Lz, Ly, Lx = mask.shape
    c = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
         (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1), (1, 0, -1),
         (-1, 0, 1), (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)]
    fluid = [(x, y, z) for z in range(Lz) for y in range(Ly) for x in range(Lx)
             if mask[z, y, x] == 0]
    index = {p: k for k, p in enumerate(fluid)}
    Nf = len(fluid)
    nbr = np.full((18, Nf), -1, np.int64)
    bb = np.zeros(Nf, np.int64)
    links = np.zeros(19, np.int64)
    for k, (x, y, z) in enumerate(fluid):
        for i in range(1, 19):
            src = ((x - c[i][0]) % Lx, (y - c[i][1]) % Ly, (z - c[i][2]) % Lz)
            if src in index:
                nbr[i - 1, k] = index[src]
            else:
                bb[k] |= 1 << i
                links[i] += 1
    fidx = [x + Lx * (y + Ly * z) for (x, y, z) in fluid]
    return np.array(fidx), nbr, bb, links


@pytest.mark.parametrize("dims,frac,seed", [((4, 4, 4), 0.3, 1), ((5, 3, 4), 0.5, 2),
                                            ((6, 6, 6), 0.2, 3), ((1, 7, 5), 0.3, 4),
                                            ((3, 1, 1), 0.0, 5), ((4, 4, 4), 1.0, 6)])
def test_links_brute_force(ora, geom, dims, frac, seed):
    mask = geom.random_mask(dims, frac, seed)
    fi, nbr, bb, lk = ora.links(mask)
    bfi, bnbr, bbb, blk = _brute_links(mask)
    assert np.array_equal(fi, bfi)
    assert np.array_equal(nbr, bnbr)
    assert np.array_equal(bb.astype(np.int64), bbb)
    assert np.array_equal(lk, blk)
    _, _, opp = ora.lattice()
    assert all(lk[i] == lk[opp[i]] for i in range(19))


def test_unit_conversion_worked_example():
    """Sec. 4.3: 5.6426 l.u. at 7 um voxels is 280,151 mD."""
    from paper_1902_11193_gb300.units import darcy_from_lattice

    (k_lb, dx, k_mD), = golden("sphere_pack_units.txt")
    got = darcy_from_lattice(float(k_lb), float(dx)) * 1e3
    assert abs(got - float(k_mD)) / float(k_mD) < 5e-6


def test_splitmix64_reference_vector(geom):
    want = [int(r[0]) for r in golden("splitmix64_seed1234567.txt")]
    assert [int(v) for v in geom.splitmix64(1234567, 5)] == want


@pytest.mark.parametrize("st,tau,lam", [("B", 0.7, 3 / 16), ("B", 1.3, 3 / 16), ("E", 0.9, 3 / 8),
                                        ("E", 1.6, 1 / 64), ("SRT", 0.8, 3 / 16)])
@pytest.mark.parametrize("linear", [False, True])
def test_trt_link_form_equals_mrt(ora, st, tau, lam, linear):
    """Sets with one even and one odd rate: the link-basis TRT collision is the
    MRT collision (Sec. 2.2), state by state."""
    s = ora.rates(st, tau, lam)
    assert s[1] == s[2] == s[9] == s[10] and s[4] == s[16]
    rng = np.random.default_rng(7)
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    for _ in range(20):
        f = w * (1 + 0.05 * rng.standard_normal(19))
        F = 1e-3 * rng.standard_normal(3)
        want = ora.collide(f, s, F, linear)
        got = ora.trt_collide(f, s[9], s[4], F, linear)
        assert np.abs(got - want).max() <= 1e-15


def test_trt_link_form_differs_for_mrt_only_sets(ora):
    """Set D has two odd rates: the single-odd-rate link form cannot express it."""
    s = ora.rates("D", 1.0)
    f = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12) * (1 + 0.05 * np.sin(np.arange(19)))
    got = ora.trt_collide(f, s[9], s[4], [1e-4, 0, 0])
    assert np.abs(got - ora.collide(f, s, [1e-4, 0, 0])).max() > 1e-6
