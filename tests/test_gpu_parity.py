"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Bars: link tables and counts bit-exact; FP64 populations and velocities
within 1e-12 of the oracle's deviations from rest at equal step counts; FP64
permeability within 1e-10; FP32-shifted permeability within 1e-5 of the FP64
oracle; the three layouts bitwise equal to each other in FP64 and FP32 (same
arithmetic, different addresses).  FP16 storage errors are reported.
"""
import numpy as np
import pytest

from gpu_util import OPP, W, dev_err, random_state, sample_nodes, upstream_nodes

pytestmark = pytest.mark.gpu

F3 = (1e-4, 2e-5, -1e-5)
LAYOUTS = ["ab", "aa", "sparse"]


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
        "random_ragged": geom.random_mask((20, 17, 13), 0.35, seed=11),  # 4420 nodes
        "sc32": geom.sphere_array(32, "sc", r=12),
        "boolean48": geom.boolean(48, 6, 0.35, seed=1902_11193 + 3)[0],
        "slit": geom.slit(9, 2, Lx=1, Lz=1),
        "tiny": geom.random_mask((3, 4, 5), 0.3, seed=2),
    }


# ------------------------------------------------------------------ structure

@pytest.mark.parametrize("name", ["random_ragged", "sc32", "boolean48", "slit", "tiny"])
def test_link_tables_bit_exact(L, ora, geom, name):
    mask = _masks(geom)[name]
    fi, nbr, bb, links = ora.links(mask)
    for layout in LAYOUTS:
        S = L.LBMSolver(mask, "B", 1.0, layout=layout, precision="fp32")
        nf, lk = S.link_counts()
        assert nf == len(fi)
        assert np.array_equal(lk, links)
        if layout == "sparse":
            gfi, gnbr, gbb = S.sparse_tables()
            assert np.array_equal(gfi, fi)
            assert np.array_equal(gnbr, nbr)
            assert np.array_equal(gbb, bb)
        S.close()


# ------------------------------------------------------------- FP64 stepping

@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("st,lam", [("A", 0.2), ("B", 0.2), ("C", 0.2), ("D", 0.2),
                                    ("E", 1 / 64), ("E", 3 / 8), ("SRT", 0.2)])
@pytest.mark.parametrize("linear", [False, True])
def test_fp64_steps_match_oracle(L, ora, geom, layout, st, lam, linear):
    mask = _masks(geom)["random_ragged"]
    f0 = random_state(mask, 1e-2, seed=5)
    tau = 0.8
    S = L.LBMSolver(mask, st, tau, lam, F3, layout=layout, precision="fp64", linear_eq=linear)
    S.set_populations(f0)
    O = ora.Solver(mask, ora.rates(st, tau, lam), F3, linear=linear)
    O.set_f(f0)
    assert dev_err(S.get_populations(), O.get_f()) <= 1e-15
    # The oracle carries unshifted f (up to 1/3, rounding 3.7e-17 per
    # operation) while these random states deviate by ~1e-3 from rest, so one
    # oracle rounding is ~1e-14 of the deviation scale; ~100 dependent
    # operations per update over <= 7 steps bound the gap by 1e-11.
    for n in (6, 1):  # compare after an even and an odd number of steps
        S.step(n)
        O.step(n)
        assert dev_err(S.get_populations(), O.get_f()) <= 1e-11
        ug, uo = S.velocity(), O.velocity()
        assert np.abs(ug - uo).max() <= 1e-11 * np.abs(uo).max()
        Ug, Uo = S.mean_velocity(), O.mean_velocity()
        assert np.abs(Ug - Uo).max() <= 1e-11 * np.abs(Uo).max()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_layouts_bitwise_equal(L, geom, precision):
    mask = _masks(geom)["boolean48"]
    f0 = random_state(mask, 1e-3, seed=9)
    outs = []
    for layout in LAYOUTS:
        for bs in (256, 128):
            S = L.LBMSolver(mask, "D", 0.9, force=F3, layout=layout, precision=precision,
                            block_size=bs)
            S.set_populations(f0)
            S.step(5)
            outs.append(S.get_populations())
            S.close()
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


# --------------------------------------------------- permeability, config 1

@pytest.fixture(scope="module")
def config1(ora, geom):
    """32^3 simple-cubic cell, centred sphere r = 12, Set E(3/16), tau = 1,
    F = 1e-6 along x, stopping rule 1e-9 evaluated every step."""
    mask = geom.sphere_array(32, "sc", r=12)
    O = ora.Solver(mask, ora.rates("E", 1.0, 3 / 16), [1e-6, 0, 0])
    rc, steps, U = O.run_to_convergence(1e-9, K=1, max_steps=100000)
    assert rc == 0
    return mask, steps, O.permeability(1.0)[0], O.velocity()


@pytest.mark.parametrize("layout", LAYOUTS)
def test_config1_fp64_permeability(L, config1, layout):
    mask, steps, k_ora, u_ora = config1
    S = L.LBMSolver(mask, "E", 1.0, 3 / 16, (1e-6, 0, 0), precision="fp64", layout=layout,
                    check_interval=1)
    rc, st = S.run_to_convergence(1e-9)
    assert rc == 0
    assert abs(st - steps) <= 1
    if st != steps:  # stop step off by one: compare at the oracle's step
        S = L.LBMSolver(mask, "E", 1.0, 3 / 16, (1e-6, 0, 0), precision="fp64", layout=layout)
        S.step(steps)
    k = S.permeability()[0]
    assert abs(k - k_ora) <= 1e-10 * abs(k_ora)
    u = S.velocity()
    # 1e-12 relative, plus the oracle's own rounding floor: it stores
    # unshifted f (<= 1/3, 3.7e-17 per rounding) and sums ten of them for a
    # velocity component, ~4e-16 absolute (3.8e-16 measured here, where
    # |u| <= 3.6e-4); the GPU stores deviations from rest and is finer.
    assert np.abs(u - u_ora).max() <= 1e-12 * np.abs(u_ora).max() + 1e-15


# ------------------------------- FP64 on Boolean media and sphere arrays

# (mask recipe, set, Lambda, tau, stopping rule, K).  The Boolean media follow
# the adjoint workload's recipe (r = 6, porosity 0.35) at 48^3 and 64^3 and
# need the two-step-mean rule (thin gaps); the BCC and FCC cells converge
# under the paper's per-step rule.  The drive F = 1e-4 puts the largest
# velocity near 1e-3, so that 1e-12 of it stays above the oracle's own
# rounding floor (it stores unshifted f <= 1/3: about 4e-16 per velocity).
FP64_CASES = {
    "boolean48": (lambda g: g.boolean(48, 6, 0.35, seed=1902_11193 + 3)[0], "B", 3 / 16, 1.0, 1, 10),
    "boolean64": (lambda g: g.boolean(64, 6, 0.35, seed=1902_11193 + 3)[0], "D", 3 / 16, 0.8, 1, 10),
    "bcc24": (lambda g: g.sphere_array(24, "bcc", c=0.3), "E", 3 / 8, 1.2, 0, 1),
    "fcc24": (lambda g: g.sphere_array(24, "fcc", c=0.3), "C", 3 / 16, 0.9, 0, 1),
}
F_BIG = (1e-4, 0.0, 0.0)
_fp64_cache = {}


def _oracle_converged(ora, geom, name):
    """The oracle run to its stopping rule (tol 1e-9): mask, stop step,
    permeability and velocity field at that step."""
    if name not in _fp64_cache:
        mk, st, lam, tau, rule, K = FP64_CASES[name]
        mask = mk(geom)
        O = ora.Solver(mask, ora.rates(st, tau, lam), list(F_BIG))
        rc, steps, _ = O.run_to_convergence(1e-9, K=K, max_steps=60000, rule=rule)
        assert rc == 0
        _fp64_cache[name] = (mask, steps, O.permeability(tau)[0], O.velocity())
        O.close()
    return _fp64_cache[name]


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("name", list(FP64_CASES))
def test_fp64_converged_matches_oracle(L, ora, geom, name, layout):
    """FP64 GPU against the FP64 oracle at the oracle's stop step: the same
    stop step (within one check interval), the velocity field within 1e-12
    of its largest component (plus the oracle's 1e-15 floor), k within
    1e-10 (eqs. perm_calc and convergence, Sec. 2.5)."""
    mask, steps, k_ora, u_ora = _oracle_converged(ora, geom, name)
    _, st, lam, tau, rule, K = FP64_CASES[name]
    S = L.LBMSolver(mask, st, tau, lam, F_BIG, precision="fp64", layout=layout,
                    check_interval=K, stop_rule=rule, max_steps=60000)
    rc, st_gpu = S.run_to_convergence(1e-9)
    assert rc == 0
    assert abs(st_gpu - steps) <= K
    S.close()
    S = L.LBMSolver(mask, st, tau, lam, F_BIG, precision="fp64", layout=layout)
    S.step(steps)
    k = S.permeability()[0]
    assert abs(k - k_ora) <= 1e-10 * abs(k_ora)
    u = S.velocity()
    assert np.abs(u - u_ora).max() <= 1e-12 * np.abs(u_ora).max() + 1e-15
    S.close()


# ----------------------------------------------- 64-bit population offsets

@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
@pytest.mark.parametrize("name", ["random_ragged", "boolean48"])
def test_wide_offsets_bitwise_equal(L, ora, geom, name, precision):
    """The sparse kernels' 64-bit-offset instantiations (taken on their own
    when 19 N_f >= 2^32) forced on small lattices: populations, the mean
    velocity and the measuring steps' stopping-rule measure are bitwise
    those of the 32-bit path; FP64 also matches the oracle."""
    mask = _masks(geom)[name]
    f0 = random_state(mask, 1e-3, seed=21)
    out = []
    for width in (0, 64):
        S = L.LBMSolver(mask, "D", 0.9, force=F3, layout="sparse", precision=precision,
                        index_width=width, check_interval=5, max_steps=17)
        S.set_populations(f0)
        S.step(7)
        f7 = S.get_populations()
        U7 = S.mean_velocity()
        rc, taken = S.run_to_convergence(0.0)  # three chunks with measuring steps
        assert rc == -4 and taken == 17
        out.append((f7, U7, S.get_populations(), S.converged_velocity()))
        S.close()
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)
    if precision == "fp64":
        O = ora.Solver(mask, ora.rates("D", 0.9), F3)
        O.set_f(f0)
        O.step(7)
        assert dev_err(out[1][0], O.get_f()) <= 1e-11


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
@pytest.mark.parametrize("edge", [96, 128])
def test_odd_tile_widths_bitwise_equal(L, geom, edge, precision):
    """The odd step's lean kernel takes four fluid nodes per thread while its
    grid fills every SM, else two or one.  The Boolean 96^3 medium (about
    352k fluid nodes) takes two, 128^3 (about 837k) four, the small lattices
    above one.  Each is bitwise the general kernel of the 64-bit-offset path
    over plain and measuring steps."""
    mask = geom.boolean(edge, 10, 0.40, seed=1902_11193 + 1)[0]
    f0 = random_state(mask, 1e-3, seed=23)
    out = []
    for width in (0, 64):
        S = L.LBMSolver(mask, "B", 1.0, force=F3, layout="sparse", precision=precision,
                        index_width=width, check_interval=6, max_steps=13)
        S.set_populations(f0)
        S.step(5)
        f5 = S.get_populations()
        rc, taken = S.run_to_convergence(0.0)
        assert rc == -4 and taken == 13
        out.append((f5, S.get_populations(), S.converged_velocity(), S.mean_velocity()))
        S.close()
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("linear", [False, True])
@pytest.mark.parametrize("st", ["B", "D"])
@pytest.mark.parametrize("parity", [0, 1])
def test_fp16_scaled_kernels_bitwise_equal(L, geom, parity, st, linear):
    """FP16 storage: the lean odd kernel and the even kernels collide the
    stored halves as they are, with the force scaled by 2^S and the
    quadratic terms by 2^-S, and plain even steps take adjacent node pairs
    per 32-bit word when N_f is even.  Against the general kernels of the
    64-bit-offset path, which multiply by 2^-S on load and 2^S on store:
    bitwise the same populations and measured velocities, for N_f even and
    odd, both collision forms (Set B: link-basis TRT; Set D: MRT) and the
    linear equilibrium."""
    mask = geom.boolean(48, 6, 0.35, seed=1902_11193 + 3)[0].copy()
    fluid = np.flatnonzero(mask.reshape(-1) == 0)
    if fluid.size % 2 != parity:  # one more solid voxel flips the parity
        mask.reshape(-1)[fluid[fluid.size // 2]] = 1
    assert int((mask == 0).sum()) % 2 == parity
    f0 = random_state(mask, 1e-3, seed=29)
    out = []
    for width in (0, 64):
        S = L.LBMSolver(mask, st, 0.9, force=F3, layout="sparse", precision="fp16",
                        index_width=width, check_interval=6, max_steps=13, linear_eq=linear)
        S.set_populations(f0)
        S.step(5)
        f5 = S.get_populations()
        rc, taken = S.run_to_convergence(0.0)
        assert rc == -4 and taken == 13
        out.append((f5, S.get_populations(), S.converged_velocity(), S.mean_velocity()))
        S.close()
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("layout", LAYOUTS)
def test_config1_fp32_permeability(L, config1, layout):
    mask, steps, k_ora, _ = config1
    S = L.LBMSolver(mask, "E", 1.0, 3 / 16, (1e-6, 0, 0), precision="fp32", layout=layout)
    S.step(steps)
    k = S.permeability()[0]
    err = abs(k - k_ora) / abs(k_ora)
    print(f"FP32 {layout}: k = {k:.10g}, oracle {k_ora:.10g}, rel err {err:.3e}")
    assert err <= 1e-5


def test_config1_fp16_permeability_reported(L, config1):
    mask, steps, k_ora, _ = config1
    for layout in ("aa", "sparse"):
        S = L.LBMSolver(mask, "E", 1.0, 3 / 16, (1e-6, 0, 0), precision="fp16", layout=layout)
        S.step(steps)
        k = S.permeability()[0]
        err = abs(k - k_ora) / abs(k_ora)
        print(f"FP16-storage {layout}: k = {k:.8g}, rel err {err:.3e}")
        assert err < 5e-2


# ------------------------------------------------------------- invariants

@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
@pytest.mark.parametrize("layout", LAYOUTS)
def test_rest_state_bit_exact(L, geom, precision, layout):
    mask = _masks(geom)["random_ragged"]
    S = L.LBMSolver(mask, "C", 0.7, force=(0, 0, 0), layout=layout, precision=precision)
    S.step(41)
    f = S.get_populations()
    assert np.array_equal(f, np.broadcast_to(W[:, None, None, None], f.shape))


@pytest.mark.parametrize("layout", LAYOUTS)
def test_mass_conserved_fp64(L, geom, layout):
    mask = _masks(geom)["boolean48"]
    f0 = random_state(mask, 1e-2, seed=3)
    S = L.LBMSolver(mask, "A", 0.7, force=F3, layout=layout, precision="fp64")
    S.set_populations(f0)
    m0 = f0.sum()
    S.step(300)
    assert abs(S.get_populations().sum() - m0) / m0 <= 1e-13


def test_rest_velocity_zero_force_half(L, geom):
    """At rest the shifted velocity of every fluid node is F/2 exactly."""
    mask = _masks(geom)["sc32"]
    S = L.LBMSolver(mask, "B", 1.0, force=(1e-6, 0, 0), precision="fp64")
    u = S.velocity()
    assert np.all(u[0][mask == 0] == 0.5e-6) and np.all(u[0][mask == 1] == 0.0)


# ------------------------------------------------------------- edge cases

@pytest.mark.parametrize("layout", LAYOUTS)
def test_degenerate_lattices(L, ora, layout):
    # all solid: no fluid node, zero velocity
    S = L.LBMSolver(np.ones((3, 4, 5), np.uint8), "B", 1.0, layout=layout)
    S.step(3)
    assert np.all(S.mean_velocity() == 0.0)
    # one fluid voxel whose every neighbour is itself (1x1x1 periodic lattice)
    # and one fluid voxel surrounded by solid: both match the oracle
    one = np.zeros((1, 1, 1), np.uint8)
    box = np.ones((3, 3, 3), np.uint8)
    box[1, 1, 1] = 0
    for mask in (one, box):
        S = L.LBMSolver(mask, "D", 0.9, force=F3, layout=layout, precision="fp64")
        O = ora.Solver(mask, ora.rates("D", 0.9), F3)
        S.step(9)
        O.step(9)
        assert dev_err(S.get_populations(), O.get_f()) <= 1e-11


def test_unstable_is_reported(L, geom):
    mask = _masks(geom)["sc32"]
    S = L.LBMSolver(mask, "SRT", 0.5001, force=(0.5, 0, 0), check_interval=10, max_steps=5000)
    rc, _ = S.run_to_convergence(1e-9, raise_on_failure=False)
    assert rc == -5


def test_max_steps_reported(L, geom):
    mask = _masks(geom)["sc32"]
    S = L.LBMSolver(mask, "B", 1.0, check_interval=7, max_steps=50)
    rc, steps = S.run_to_convergence(0.0)
    assert rc == -4 and steps == 50 and S.steps == 50


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
def test_checkpoint_resume_bitwise(L, geom, tmp_path, layout, precision):
    mask = _masks(geom)["boolean48"]
    A = L.LBMSolver(mask, "E", 1.2, 3 / 8, F3, layout=layout, precision=precision)
    A.step(5)  # odd: the AA patterns resume at the odd parity
    path = str(tmp_path / "ck.lbm")
    A.save(path)
    A.step(6)
    B = L.LBMSolver.load(path)
    assert B.steps == 5
    B.step(6)
    assert np.array_equal(A.get_populations(), B.get_populations())
    assert np.array_equal(A.permeability(), B.permeability())


# ------------------------------------------- full size, bench configuration

@pytest.mark.parametrize("layout,precision,warm,tol", [
    ("aa", "fp32", 3, 1e-5), ("aa", "fp32", 2, 1e-5),
    ("sparse", "fp32", 3, 1e-5), ("sparse", "fp32", 2, 1e-5),
    ("sparse", "fp16", 3, 1e-3), ("sparse", "fp16", 2, 1e-3)])
def test_512_boolean_sampled_parity(L, ora, geom, layout, precision, warm, tol):
    """512^3 Boolean medium (r = 10, porosity 0.40, Set B, tau = 1, F = 1e-6)
    in the benchmark's launch configuration: after `warm` steps, sampled
    nodes' next post-collision populations are recomputed by the oracle from
    the GPU state of their upstream neighbourhood.  warm = 3 checks an odd
    step, 2 an even one.  FP32 storage within 1e-5 of the largest deviation
    from rest; FP16 storage (the even step's node pairs, N_f being even
    here, and the odd step's scaled collision) within 1e-3: the stored halves
    round at 2^-11 of their values."""
    mask, _ = geom.boolean(512, 10, 0.40, seed=1902_11193 + 1)
    F = (1e-6, 0.0, 0.0)
    S = L.LBMSolver(mask, "B", 1.0, force=F, layout=layout, precision=precision)
    S.step(warm)
    nodes = sample_nodes(mask, 400, seed=1)
    ups = upstream_nodes(mask, nodes)
    fstar = S.get_populations_at(ups.reshape(-1)).reshape(len(nodes), 19, 19)
    s = ora.rates("B", 1.0)
    pred = np.zeros((len(nodes), 19))
    flat = mask.reshape(-1)
    for k in range(len(nodes)):
        fl = np.empty(19)
        for i in range(19):
            src = ups[k, i]
            fl[i] = fstar[k, 0, OPP[i]] if flat[src] else fstar[k, i, i]
        pred[k] = ora.collide(fl, s, F)
    S.step(1)
    got = S.get_populations_at(nodes)
    assert dev_err(got.T, pred.T) <= tol
    nf, _ = S.link_counts()
    assert nf == int((mask == 0).sum())


@pytest.mark.parametrize("precision,warm,tol", [
    ("fp32", 3, 1e-5), ("fp16", 3, 1e-3), ("fp16", 2, 1e-3)])
def test_1024_boolean_sampled_parity(L, ora, geom, precision, warm, tol):
    """The large low-porosity image: 1024^3 Boolean medium (r = 8, porosity
    0.20, Set D: the moment-space MRT collision, tau = 1, F = 1e-6), sparse,
    as the bench's 1024^3 leg runs it (19 N_f just under 2^32: 32-bit
    offsets).  Sampled nodes' next post-collision populations against the
    oracle's collision of the GPU's upstream state, as at 512^3."""
    mask, _ = geom.boolean(1024, 8, 0.20, seed=1902_11193 + 5)
    F = (1e-6, 0.0, 0.0)
    S = L.LBMSolver(mask, "D", 1.0, force=F, layout="sparse", precision=precision)
    S.step(warm)
    nodes = sample_nodes(mask, 300, seed=2)
    ups = upstream_nodes(mask, nodes)
    fstar = S.get_populations_at(ups.reshape(-1)).reshape(len(nodes), 19, 19)
    s = ora.rates("D", 1.0)
    pred = np.zeros((len(nodes), 19))
    flat = mask.reshape(-1)
    for k in range(len(nodes)):
        fl = np.empty(19)
        for i in range(19):
            fl[i] = fstar[k, 0, OPP[i]] if flat[ups[k, i]] else fstar[k, i, i]
        pred[k] = ora.collide(fl, s, F)
    S.step(1)
    got = S.get_populations_at(nodes)
    assert dev_err(got.T, pred.T) <= tol
    S.close()


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("shape", ["ragged", "x_faces"])
def test_mean_velocity_equals_exported_field_mean(L, geom, layout, precision, shape):
    """lbm_mean_velocity (float momenta, compensated sums for FP32/FP16
    storage) against the mean of the FP64 velocity-field export, on a ragged
    lattice with fluid on the x faces, after an odd and an even number of
    steps.  In the x_faces case every fluid voxel lies within four voxels of
    an x face (the channel wraps across the periodic x boundary), so the
    wrapped upstream indices carry all of the momentum.  Each component
    within 1e-7 of itself: the float per-node momenta round at ~6e-8 of
    their terms, and those roundings average out over the nodes."""
    mask = geom.random_mask((21, 18, 37), 0.3, seed=7)
    if shape == "x_faces":
        mask[:, :, 4:17] = 1
    S = L.LBMSolver(mask, "B", 0.8, force=(2e-5, -1e-5, 5e-6), precision=precision, layout=layout)
    for n in (7, 1):
        S.step(n)
        U = S.mean_velocity()
        u = S.velocity()
        Uf = np.array([u[a].sum() for a in range(3)]) / mask.size
        assert np.all(np.abs(U - Uf) <= 1e-7 * np.abs(Uf)), (U, Uf)
    S.close()
