"""The CUDA steady-state adjoint (lbm_adjoint) against the oracle's adjoint and
against central finite differences of the converged permeability.

Gradients are compared normalised: tau dk/dtau / k, Lambda dk/dLambda / k,
F dk/dF / k.  FP64 GPU vs FP64 oracle adjoint: 1e-7 (both are accurate to
~1e-8: the oracle differences the rate formulas in tau with step 1e-5).
FP32 forward + adjoint vs FP64 finite differences (step 1e-4, forward solves
converged to 1e-13 per step): 1e-4, the stated target.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

F1 = (1e-5, 0.0, 0.0)


@pytest.fixture(scope="module")
def L():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_11193_gb300 import lbm

    lbm.lib()
    return lbm


def _norm(g, k, tau, lam, F):
    return {"dtau": g["dtau"] * tau / k, "dLambda": g["dLambda"] * lam / k,
            "dLambda_q": g["dLambda_q"] * (3 / 16) / k, "dLambda_m": g["dLambda_m"] * (3 / 8) / k,
            "dF": g["dF"][0] * F[0] / k}


def _ora_grad(ora, mask, st, tau, lam, F, linear=False):
    O = ora.Solver(mask, ora.rates(st, tau, lam), F, linear=linear)
    rc, _, U = O.run_to_convergence(1e-15, K=10, max_steps=60000)
    assert rc == 0
    k = (tau - 0.5) / 3 * U[0] / F[0]
    rc, g, _ = O.adjoint(st, tau, lam, tol=1e-12)
    assert rc == 0
    g = dict(g, dF=np.array([g["dFx"], g["dFy"], g["dFz"]]))
    return k, g


def _gpu_grad(L, mask, st, tau, lam, F, precision="fp64", layout="ab", tol=1e-15, atol=1e-12,
              linear=False, rule=0):
    S = L.LBMSolver(mask, st, tau, lam, F, precision=precision, layout=layout, check_interval=10,
                    max_steps=100000, linear_eq=linear, stop_rule=rule)
    rc, steps = S.run_to_convergence(tol)
    assert rc == 0, (precision, tol, steps)
    g = S.adjoint(atol, max_iter=100000)
    assert g["residual"] <= atol, (precision, g["residual"], g["iterations"])
    return g["k"], g, S


@pytest.mark.parametrize("layout", ["ab", "aa", "sparse"])
@pytest.mark.parametrize("st,lam", [("E", 3 / 8), ("D", 3 / 16), ("A", 3 / 16), ("SRT", 3 / 16),
                                    ("C", 3 / 16)])
def test_fp64_adjoint_matches_oracle(L, ora, geom, layout, st, lam):
    mask = geom.sphere_array(10, "bcc", r=3.2)
    tau = 0.9
    ko, go = _ora_grad(ora, mask, st, tau, lam, F1)
    kg, gg, _ = _gpu_grad(L, mask, st, tau, lam, F1, layout=layout)
    assert abs(kg - ko) <= 1e-10 * abs(ko)
    no, ng = _norm(go, ko, tau, lam, F1), _norm(gg, kg, tau, lam, F1)
    for key in ("dtau", "dF"):
        assert abs(ng[key] - no[key]) < 1e-7, (key, ng[key], no[key])
    for key in ("dLambda", "dLambda_q", "dLambda_m"):
        if st in ("B", "D", "E"):
            assert abs(ng[key] - no[key]) < 1e-7, (key, ng[key], no[key])
        else:
            assert np.isnan(ng[key]) and np.isnan(no[key])
    assert np.abs(gg["dF"][1:]).max() < 1e-6 * abs(kg / F1[0])


def test_adjoint_state_errors(L, geom):
    mask = geom.sphere_array(10, "bcc", r=3.2)
    S = L.LBMSolver(mask, "B", 1.0, force=F1)
    with pytest.raises(L.LBMError) as e:
        S.adjoint()
    assert e.value.code == -7  # ENOSTATE: not converged
    S.run_to_convergence(1e-8)
    S.step(1)
    with pytest.raises(L.LBMError) as e:
        S.adjoint()
    assert e.value.code == -7
    Z = L.LBMSolver(mask, "B", 1.0, force=(0.0, 0.0, 0.0), check_interval=2, max_steps=10)
    Z.run_to_convergence(1e-3)
    with pytest.raises(L.LBMError) as e:
        Z.adjoint()
    assert e.value.code in (-1, -7)


@pytest.fixture(scope="module")
def boolean48(geom):
    """48^3 Boolean medium, sphere radius 6, porosity 0.35.  Its one- and
    two-voxel gaps carry bounceback modes of eigenvalue near -1, so every
    solve on it uses the two-step-mean stopping rule."""
    return geom.boolean(48, 6, 0.35, seed=1902_11193 + 4)[0]


def _magic_rates(L, st, tau, lam, Lq=None, Lm=None):
    """Table 2 rates of the set, with the odd rates s_q and s_m set through
    their own magic parameters where given (Set E's formula, Sec. 2.3)."""
    s = L.rates(st, tau, lam)
    if Lq is not None:
        s[[4, 6, 8]] = L.rates("E", tau, Lq)[4]
    if Lm is not None:
        s[[16, 17, 18]] = L.rates("E", tau, Lm)[16]
    return s


def _fd(L, mask, st, tau, lam, F, which, h=1e-4):
    """Central difference of the FP64 permeability at the fixed point (the
    two-step mean the stopping rule converged on, to 1e-12).  h is an
    absolute step in tau and the magic parameters, a relative one in F."""
    def k_at(t=tau, Fv=F, Lq=None, Lm=None):
        kw = dict(precision="fp64", layout="sparse", check_interval=20, max_steps=100000,
                  stop_rule=1)
        if Lq is None and Lm is None:
            S = L.LBMSolver(mask, st, t, lam, Fv, **kw)
        else:
            S = L.LBMSolver(mask, force=Fv, rates_=_magic_rates(L, st, t, lam, Lq, Lm), **kw)
        rc, _ = S.run_to_convergence(1e-12)
        assert rc == 0
        k = S.converged_permeability()[0]
        S.close()
        return k
    if which == "dtau":
        return (k_at(t=tau + h) - k_at(t=tau - h)) / (2 * h)
    if which == "dLambda":  # Sets B, E: both odd rates through one parameter
        return (k_at(Lq=lam + h, Lm=lam + h) - k_at(Lq=lam - h, Lm=lam - h)) / (2 * h)
    if which == "dLambda_q":  # Set D: Lambda_q = 3/16
        return (k_at(Lq=3 / 16 + h) - k_at(Lq=3 / 16 - h)) / (2 * h)
    if which == "dLambda_m":  # Set D: Lambda_m = 3/8
        return (k_at(Lm=3 / 8 + h) - k_at(Lm=3 / 8 - h)) / (2 * h)
    Fp, Fm = (F[0] * (1 + h), 0, 0), (F[0] * (1 - h), 0, 0)
    return (k_at(Fv=Fp) - k_at(Fv=Fm)) / (2 * h * F[0])


# the adjoint study's grid: Sets B, D, E(3/8) at tau = 0.8, 1.0, 1.3
FD_GRID = [(st, lam, tau) for st, lam in (("B", 3 / 16), ("D", 3 / 16), ("E", 3 / 8))
           for tau in (0.8, 1.0, 1.3)]


@pytest.mark.parametrize("st,lam,tau", FD_GRID)
def test_fp32_adjoint_vs_finite_differences_48(L, boolean48, st, lam, tau):
    """FP32 forward and adjoint against FP64 central differences (h = 1e-4)
    of the converged permeability, every gradient component, normalised
    (theta dk/dtheta / k) within 1e-4."""
    F = (1e-6, 0.0, 0.0)
    k, g, S = _gpu_grad(L, boolean48, st, tau, lam, F, precision="fp32", layout="sparse", tol=1e-8,
                        atol=1e-6, rule=1)
    checks = ["dtau", "dF"] + (["dLambda_q", "dLambda_m"] if st == "D" else ["dLambda"])
    for key in checks:
        fd = _fd(L, boolean48, st, tau, lam, F, key)
        scale = {"dtau": tau, "dLambda": lam, "dLambda_q": 3 / 16, "dLambda_m": 3 / 8,
                 "dF": F[0]}[key]
        adj = g["dF"][0] if key == "dF" else g[key]
        err = abs(adj * scale / k - fd * scale / k)
        print(f"{st} tau={tau} {key}: adjoint {adj * scale / k:+.6e} fd {fd * scale / k:+.6e}"
              f" err {err:.2e}")
        assert err < 1e-4
    S.close()


def test_adjoint_boolean_vs_oracle(L, ora, boolean48):
    """The 48^3 Boolean medium of the adjoint study (r = 6, porosity 0.35),
    Set D at tau = 1: FP64 and FP32 GPU adjoints against the oracle's
    adjoint (about a minute of host time)."""
    mask = boolean48
    st, tau, lam = "D", 1.0, 3 / 16
    F = (1e-6, 0.0, 0.0)
    O = ora.Solver(mask, ora.rates(st, tau, lam), F)
    rc, _, U = O.run_to_convergence(1e-11, K=10, max_steps=60000, rule=1)
    assert rc == 0
    rc, go, _ = O.adjoint(st, tau, lam, tol=1e-9, max_iter=60000)
    assert rc == 0
    go = dict(go, dF=np.array([go["dFx"], go["dFy"], go["dFz"]]))
    ko = (tau - 0.5) / 3 * U[0] / F[0]
    no = _norm(go, ko, tau, lam, F)
    kg, gg, _ = _gpu_grad(L, mask, st, tau, lam, F, precision="fp64", layout="sparse", tol=1e-11,
                          atol=1e-9, rule=1)
    ng = _norm(gg, kg, tau, lam, F)
    k3, g3, _ = _gpu_grad(L, mask, st, tau, lam, F, precision="fp32", layout="sparse",
                          tol=1e-8, atol=1e-6, rule=1)
    n3 = _norm(g3, k3, tau, lam, F)
    assert abs(kg - ko) <= 1e-9 * abs(ko)
    for key in ("dtau", "dLambda_q", "dLambda_m", "dF"):
        print(f"{key}: oracle {no[key]:+.8e} fp64 {ng[key]:+.8e} fp32 {n3[key]:+.8e}")
        assert abs(ng[key] - no[key]) < 1e-6
        assert abs(n3[key] - no[key]) < 1e-4


def test_autograd_function(L, geom):
    import torch

    from paper_1902_11193_gb300.autograd import permeability

    mask = geom.sphere_array(10, "bcc", r=3.2)
    tau = torch.tensor(0.9, dtype=torch.float64, requires_grad=True)
    lam = torch.tensor(3 / 8, dtype=torch.float64, requires_grad=True)
    F = torch.tensor(F1, dtype=torch.float64, requires_grad=True)
    k = permeability(mask, tau, lam, F, set_="E", tol=1e-14, adjoint_tol=1e-12,
                     precision="fp64", check_interval=10)
    k.backward()
    _, g, _ = _gpu_grad(L, mask, "E", 0.9, 3 / 8, F1)
    assert abs(k.item() - g["k"]) <= 1e-12 * abs(g["k"])
    assert abs(tau.grad.item() - g["dtau"]) <= 1e-9 * abs(g["k"])
    assert abs(lam.grad.item() - g["dLambda"]) <= 1e-9 * abs(g["dLambda"]) + 1e-12
    assert np.allclose(F.grad.numpy(), g["dF"], rtol=1e-9, atol=1e-6)


@pytest.mark.parametrize("layout", ["ab", "aa", "sparse"])
@pytest.mark.parametrize("n", [1, 7, 25])
def test_transient_adjoint_fp64_matches_oracle(L, ora, geom, layout, n):
    """Checkpointed reverse sweep (segments of ceil(sqrt(n)) steps, the last
    one shorter for n = 7) against the oracle's store-everything recursion."""
    mask = geom.sphere_array(8, "bcc", r=2.4)
    tau, F = 0.9, (1e-5, 2e-6, 0.0)
    O = ora.Solver(mask, ora.rates("D", tau), list(F))
    rc, go = O.adjoint_transient("D", tau, n=n)
    assert rc == 0
    S = L.LBMSolver(mask, "D", tau, force=F, precision="fp64", layout=layout)
    g = S.adjoint_transient(n)
    assert S.steps == n and g["iterations"] == n
    k = O.permeability(tau)[0]
    assert abs(g["k"] / k - 1) <= 1e-11
    # the oracle differences the rates in tau and Lambda with step 1e-5: its
    # per-step terms carry ~1e-10 relative truncation error
    for key, sc in (("dtau", tau), ("dLambda_q", 3 / 16), ("dLambda_m", 3 / 8)):
        assert abs(g[key] - go[key]) * sc <= 1e-8 * abs(k), key
    for a, key in enumerate(("dFx", "dFy")):
        assert abs(g["dF"][a] - go[key]) * F[0] <= 1e-9 * abs(k), key
    # the context ends where a plain n-step run ends
    P = L.LBMSolver(mask, "D", tau, force=F, precision="fp64", layout=layout)
    P.step(n)
    assert np.array_equal(S.velocity(), P.velocity())


def test_transient_adjoint_fp32_close_to_fp64(L, geom, boolean48):
    tau, F, n = 1.0, (1e-6, 0.0, 0.0), 300
    out = {}
    for prec in ("fp64", "fp32"):
        S = L.LBMSolver(boolean48, "B", tau, force=F, precision=prec, layout="sparse")
        out[prec] = S.adjoint_transient(n)
    k = out["fp64"]["k"]
    for key, sc in (("dtau", tau), ("dLambda", 3 / 16)):
        assert abs(out["fp32"][key] - out["fp64"][key]) * sc <= 1e-4 * abs(k), key


def test_transient_adjoint_tends_to_steady(L, geom):
    mask = geom.sphere_array(10, "bcc", r=3.2)
    tau, F = 1.4, (1e-6, 0.0, 0.0)
    A = L.LBMSolver(mask, "B", tau, force=F, precision="fp64", layout="aa", check_interval=10)
    g_tr = A.adjoint_transient(800)
    B = L.LBMSolver(mask, "B", tau, force=F, precision="fp64", layout="aa", check_interval=10)
    rc, _ = B.run_to_convergence(1e-14)
    assert rc == 0
    g_st = B.adjoint(1e-13, max_iter=200000)
    k = g_st["k"]
    for key, sc in (("dtau", tau), ("dLambda", 3 / 16)):
        assert abs(g_tr[key] - g_st[key]) * sc <= 1e-8 * abs(k), key


def test_transient_autograd_matches_differences(L, geom):
    """transient_permeability's gradients against central differences of GPU
    FP64 runs of n steps from rest."""
    import torch

    from paper_1902_11193_gb300.autograd import transient_permeability

    mask = geom.sphere_array(12, "bcc", c=0.3)
    n, t0, l0, f0 = 60, 0.9, 3 / 8, 1e-5
    tau = torch.tensor(t0, dtype=torch.float64, requires_grad=True)
    lam = torch.tensor(l0, dtype=torch.float64, requires_grad=True)
    F = torch.tensor([f0, 0.0, 0.0], dtype=torch.float64, requires_grad=True)
    k = transient_permeability(mask, tau, lam, F, n, set_="E", precision="fp64", layout="aa")
    k.backward()

    def kn(t, lm, fx):
        S = L.LBMSolver(mask, "E", t, lm, (fx, 0.0, 0.0), precision="fp64", layout="aa")
        S.step(n)
        out = S.permeability()[0]
        S.close()
        return out

    kv = float(k.detach())
    assert abs(kv / kn(t0, l0, f0) - 1) <= 1e-12
    h = 1e-4
    fd_tau = (kn(t0 + h, l0, f0) - kn(t0 - h, l0, f0)) / (2 * h)
    fd_lam = (kn(t0, l0 + h, f0) - kn(t0, l0 - h, f0)) / (2 * h)
    fd_F = (kn(t0, l0, f0 * (1 + h)) - kn(t0, l0, f0 * (1 - h))) / (2 * h * f0)
    scale = abs(kv)
    assert abs(float(tau.grad) - fd_tau) * t0 <= 1e-6 * scale
    assert abs(float(lam.grad) - fd_lam) * l0 <= 1e-6 * scale
    assert abs(float(F.grad[0]) - fd_F) * f0 <= 1e-6 * scale


def test_transient_adjoint_contract(L, geom):
    mask = geom.sphere_array(10, "bcc", r=3.2)
    S = L.LBMSolver(mask, "B", 1.0, force=(1e-6, 0, 0), precision="fp64", layout="ab")
    for n in (0, -3):
        with pytest.raises(L.LBMError):
            S.adjoint_transient(n)
    Z = L.LBMSolver(mask, "B", 1.0, force=(0, 0, 0), precision="fp64", layout="ab")
    with pytest.raises(L.LBMError):  # no drive, no derivative of k along it
        Z.adjoint_transient(5)
    for kw in (dict(bounceback="fullway"), dict(symmetry="y")):
        X = L.LBMSolver(mask, "B", 1.0, force=(1e-6, 0, 0), precision="fp64", layout="ab", **kw)
        with pytest.raises(L.LBMError):
            X.adjoint_transient(5)
        X.close()
    assert S.steps == 0  # refused calls leave the context where it was


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_sparse_adjoint_on_fluid_x_faces(L, geom, precision):
    """Fluid at both x faces of the first and last rows: the x-moving
    upstream indices of those nodes wrap around the periodic box (at the
    ends of the fluid list the unwrapped formula would point outside it).
    The sparse adjoint (steady and transient) must equal the dense one."""
    mask = np.zeros((12, 10, 16), np.uint8)
    mask[3:9, 3:7, 5:11] = 1  # a solid block in the middle; every face fluid
    out = {}
    for layout in ("aa", "sparse"):
        S = L.LBMSolver(mask, "B", 0.9, force=(1e-5, 2e-6, 0.0), precision=precision,
                        layout=layout, check_interval=10, stop_rule=1)
        rc, _ = S.run_to_convergence(1e-10 if precision == "fp64" else 1e-7)
        assert rc == 0
        g = S.adjoint(1e-12 if precision == "fp64" else 1e-6)
        gt = S.adjoint_transient(9)
        out[layout] = (g, gt)
        S.close()
    tol = 1e-10 if precision == "fp64" else 1e-4
    for a, b in zip(out["aa"], out["sparse"]):
        for key in ("dtau", "dLambda_q", "dLambda_m"):
            assert abs(a[key] - b[key]) <= tol * (abs(a[key]) + abs(a["k"])), key
        assert np.abs(a["dF"] - b["dF"]).max() <= tol * (np.abs(a["dF"]).max() + abs(a["k"]))
