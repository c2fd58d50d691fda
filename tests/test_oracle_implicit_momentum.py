"""Pins of the oracle's fully implicit variable-viscosity momentum: the whole
stress of Eq. 4.1, div(2 eta(phi) D(v)), by Crank-Nicolson with u and v
coupled (the eta_bar split of Eq. 4.2 replaced).  CPU only.

  * div(2 eta D(v)) against its sympy form at order 2 (§4 "second order
    accuracy"), non-constant eta, a velocity that is not divergence-free;
  * the matrix is symmetric and rho/dt bounds its spectrum from below on
    the fields that vanish on the walls (the viscous form is positive
    semi-definite), at a 10:1 and at the paper's 4.3e5:1 viscosity ratio;
  * Jacobi-CG equals dense LU;
  * a shear wave u = sin(pi l y) (v = 0, uniform eta) decays by exactly the
    Crank-Nicolson factor of the discrete eigenvalue of d/dy(eta d/dy);
  * planted mistakes each fail a pin."""
import math

import numpy as np
import pytest
import sympy as sp

from oracle import cahn_oracle as O
from paper_1811_11842_gb300 import inputs as I

LX, LY = 2.0, 1.0
X_, Y_ = sp.symbols("x y")
K1 = 2 * sp.pi * X_ / LX
PY = sp.pi * Y_ / LY


def _num(expr):
    f = sp.lambdify((X_, Y_), expr, "numpy")
    return lambda X, Y: np.broadcast_to(f(X, Y), X.shape).astype(np.float64)


def _coords(g):
    return np.meshgrid(np.arange(g.nx) * g.hx, np.arange(g.ny + 1) * g.hy)


def _rate(errs):
    return [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


def check_stress_mms(Om):
    eta = 3 + sp.Rational(6, 5) * sp.sin(K1 + sp.Rational(3, 10)) * sp.cos(PY) \
        + sp.Rational(1, 2) * sp.cos(2 * K1) * sp.cos(2 * PY)
    u = sp.cos(K1) * sp.sin(PY) + sp.Rational(3, 10) * sp.sin(2 * K1 + sp.Rational(1, 2)) * sp.sin(2 * PY)
    v = sp.Rational(2, 5) * sp.sin(K1 + sp.Rational(1, 5)) * sp.sin(PY) ** 2 + sp.Rational(1, 5) * sp.cos(K1) * sp.sin(2 * PY)
    dxx, dyy = sp.diff(u, X_), sp.diff(v, Y_)
    dxy = (sp.diff(u, Y_) + sp.diff(v, X_)) / 2
    eu = sp.diff(2 * eta * dxx, X_) + sp.diff(2 * eta * dxy, Y_)
    ev = sp.diff(2 * eta * dxy, X_) + sp.diff(2 * eta * dyy, Y_)
    f = {k: _num(e) for k, e in dict(eta=eta, u=u, v=v, eu=eu, ev=ev).items()}
    errs = []
    for n in (32, 64, 128):
        g = O.Grid(n, n, LX, LY)
        X, Y = _coords(g)
        val = {k: fn(X, Y) for k, fn in f.items()}
        for k in ("u", "v"):
            val[k][0] = val[k][-1] = 0.0
        tu, tv = Om.viscous_stress_div(g, val["eta"], val["u"], val["v"])
        err = max(np.max(np.abs(tu - val["eu"])[1:-1]), np.max(np.abs(tv - val["ev"])[1:-1]))
        errs.append(err / max(np.max(np.abs(val["eu"])), np.max(np.abs(val["ev"]))))
        assert np.all(tu[[0, -1]] == 0.0) and np.all(tv[[0, -1]] == 0.0)
    assert all(1.85 < r < 2.2 for r in _rate(errs)), (errs, _rate(errs))


def _interior_matrix(Om, prm, g, eta):
    ny1 = g.ny + 1
    shape = (2 * ny1, g.nx)

    def apply(x):
        yu, yv = Om.visc_apply(prm, g, eta, x[:ny1], x[ny1:])
        return np.concatenate([yu, yv], axis=0)

    A = Om.assemble(apply, shape)
    rows = np.ones(shape, dtype=bool)
    for r in (0, g.ny, ny1, ny1 + g.ny):
        rows[r] = False
    keep = rows.ravel()
    return A[np.ix_(keep, keep)]


def check_symmetric_positive(Om):
    for eb in (10.0, 1.0 / 2.33e-9):
        prm = I.Params(nx=12, ny=10, lx=2.0, ly=1.0, dt=1e-3, eta_water=1.0, eta_biofilm=eb,
                       momentum=1)
        if eb > 100:
            prm = prm.replace(eta_water=1.0 / 9.98e-4, dt=0.1)
        g = Om.grid_of(prm)
        rng = np.random.default_rng(5)
        phi = 0.2 + 0.6 * rng.random(g.shape)
        eta = Om.viscosity(prm, phi)
        A = _interior_matrix(Om, prm, g, eta)
        assert np.max(np.abs(A - A.T)) <= 1e-13 * np.max(np.abs(A)), eb
        lam = np.linalg.eigvalsh(0.5 * (A + A.T))
        c0 = prm.rho_water / prm.dt
        assert lam[0] >= c0 * (1 - 1e-9), (eb, lam[0], c0)


def check_cg_vs_lu(Om):
    prm = I.Params(nx=16, ny=12, lx=2.0, ly=1.0, dt=1e-3, eta_water=1.0, eta_biofilm=10.0,
                   momentum=1, flow_mode=I.FLOW_SHEAR, u_max=0.3)
    g = Om.grid_of(prm)
    rng = np.random.default_rng(8)
    eta = Om.viscosity(prm, 0.2 + 0.6 * rng.random(g.shape))
    bu, bv = rng.standard_normal(g.shape), rng.standard_normal(g.shape)
    ul, vl = Om.visc_solve(prm, g, eta, bu, bv, method="lu")
    uc, vc = Om.visc_solve(prm, g, eta, bu, bv)
    assert np.max(np.abs(uc - ul)) <= 1e-12 * np.max(np.abs(ul))
    assert np.max(np.abs(vc - vl)) <= 1e-12 * np.max(np.abs(vl))


def check_shear_wave_decay(Om):
    """One implicit step of u = sin(pi l y / Ly), v = 0 in uniform phi: no
    convection, no capillary force, divergence-free, so p = 0 and
    u^{n+1} = (c0 - lam/2) / (c0 + lam/2) u^n, lam = eta (4/hy^2) sin^2(pi l / 2 ny)."""
    prm = I.Params(nx=8, ny=16, lx=2.0, ly=1.0, dt=1e-2, eta_water=2.0, eta_biofilm=2.0,
                   momentum=1, flow_mode=I.FLOW_SHEAR, u_max=0.0)
    g = Om.grid_of(prm)
    _, Y = _coords(g)
    for l in (1, 3):
        u = np.sin(math.pi * l * Y / g.ly)
        u[0] = u[-1] = 0.0
        z = np.zeros(g.shape)
        st = Om.init_state(prm, 0.4 * np.ones(g.shape), u, z, z)
        out = Om.step(prm, st)
        lam = 2.0 * 4.0 / g.hy ** 2 * math.sin(math.pi * l / (2 * g.ny)) ** 2
        c0 = 1.0 / prm.dt
        fac = (c0 - 0.5 * lam) / (c0 + 0.5 * lam)
        assert np.max(np.abs(out.u - fac * u)) <= 1e-12, (l, np.max(np.abs(out.u - fac * u)))
        assert np.max(np.abs(out.v)) <= 1e-12 and np.max(np.abs(out.p)) <= 1e-12


CHECKS = [check_stress_mms, check_symmetric_positive, check_cg_vs_lu, check_shear_wave_decay]


@pytest.mark.parametrize("check", CHECKS, ids=lambda c: c.__name__)
def test_implicit_momentum_pin(check):
    check(O)


def test_poiseuille_steady_with_implicit_momentum():
    prm = I.Params(nx=32, ny=16, eta_water=2.0, eta_biofilm=2.0, u_max=1.0, dt=1e-3, momentum=1)
    u0, v0, p0 = I.initial_velocity(prm)
    st = O.run(prm, 0.4 * np.ones_like(u0), u0, v0, p0, 5)
    assert np.max(np.abs(st.u - u0)) < 1e-11
    assert np.max(np.abs(st.v)) < 1e-12 and np.max(np.abs(st.p)) < 1e-12


_ORIG = O.viscous_stress_div


def _no_cross(g, eta, u, v):
    tu = O.dxx_face(g, 2.0 * eta, u) + O.dyy_face(g, eta, u)
    tv = O.dxx_face(g, eta, v) + O.dyy_face(g, 2.0 * eta, v)
    tu[[0, -1]] = 0.0
    tv[[0, -1]] = 0.0
    return tu, tv


def _no_two(g, eta, u, v):
    tu = O.dxx_face(g, eta, u) + O.dyy_face(g, eta, u) + O.dy_c(g, eta * O.dx_c(g, v))
    tv = O.dx_c(g, eta * O.dy_c(g, u)) + O.dxx_face(g, eta, v) + O.dyy_face(g, eta, v)
    tu[[0, -1]] = 0.0
    tv[[0, -1]] = 0.0
    return tu, tv


def _cross_swapped(g, eta, u, v):
    tu = O.dxx_face(g, 2.0 * eta, u) + O.dyy_face(g, eta, u) + O.dx_c(g, eta * O.dy_c(g, v))
    tv = O.dy_c(g, eta * O.dx_c(g, u)) + O.dxx_face(g, eta, v) + O.dyy_face(g, 2.0 * eta, v)
    tu[[0, -1]] = 0.0
    tv[[0, -1]] = 0.0
    return tu, tv


def _full_weight(prm, g, eta, u, v):
    c0 = O.rho0(prm) / prm.dt
    tu, tv = _ORIG(g, eta, u, v)
    return c0 * u - tu, c0 * v - tv


MUTANTS = {
    "cross derivatives dropped": ("viscous_stress_div", _no_cross),
    "normal stress without the factor 2": ("viscous_stress_div", _no_two),
    "cross derivatives in the other order": ("viscous_stress_div", _cross_swapped),
    "Crank-Nicolson weight 1 in the matrix": ("visc_apply", _full_weight),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, monkeypatch):
    attr, bad = MUTANTS[name]
    monkeypatch.setattr(O, attr, bad)
    failed = []
    for check in CHECKS:
        try:
            check(O)
        except AssertionError:
            failed.append(check.__name__)
    assert failed, f"planted mistake {name} passed every pin"
