"""Pins of the oracle's momentum right-hand side (Eq. 4.1-4.3) to continuous
forms outside the oracle: each term against its sympy derivative at the
nodes, with the observed order 2 of §4 ("second order accuracy") over three
grids.  CPU only.

The fields are smooth, periodic in x, with zero wall-normal derivative of
phi on the walls (Eq. 4.6) and no-slip velocities (u = v = 0 on y = 0 and
y = Ly), so every difference the oracle takes near a wall is a central
difference of exact values and the error is O(h^2) up to the walls.  The
time levels differ (phi^{n+1} != phi^n, u^{n-1} != u^n), so a term taken at
the wrong level leaves an O(1) error.

Terms:
  convection      rho (v* . grad) u*, rho (v* . grad) v*,  v* = (3 v^n - v^{n-1})/2
  capillary       -Gamma div(grad phi (x) grad phi) at phi^{n+1/2} (Eq. 4.1)
  viscous         eta_bar/2 Lap u^n (the explicit Crank-Nicolson half) and
                  the explicit remainder div(eta' grad v*) + (grad v*)^T grad eta',
                  eta' = eta(phi^{n+1/2}) - eta_bar; for a divergence-free v*
                  this equals div(2 eta' D(v*)), the stress of Eq. 4.1, which
                  a second check compares against directly.

The bottom of the file plants one mistake at a time in the oracle (on the
CPU, for one test) and requires a pin to fail."""
import dataclasses
import math

import numpy as np
import pytest
import sympy as sp

from oracle import cahn_oracle as O
from paper_1811_11842_gb300 import inputs as I

LX, LY = 2.0, 1.0
X_, Y_ = sp.symbols("x y")
K1 = 2 * sp.pi * X_ / LX          # fundamental x mode
PY = sp.pi * Y_ / LY


def _num(expr):
    f = sp.lambdify((X_, Y_), expr, "numpy")
    return lambda X, Y: np.broadcast_to(f(X, Y), X.shape).astype(np.float64)


def _coords(g):
    x = np.arange(g.nx) * g.hx
    y = np.arange(g.ny + 1) * g.hy
    return np.meshgrid(x, y)


def _rate(errs):
    return [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


# manufactured levels -------------------------------------------------------

def _phi_levels():
    """phi^n and phi^{n+1}: Neumann (cos(m pi y)) in y, values in (0.2, 0.8)."""
    phi_n = (sp.Rational(1, 2) + sp.Rational(1, 5) * sp.cos(K1 + sp.Rational(3, 10)) * sp.cos(PY)
             + sp.Rational(1, 10) * sp.cos(2 * K1) * sp.cos(2 * PY))
    phi_1 = phi_n + sp.Rational(1, 20) * sp.sin(K1) * sp.cos(PY) \
        + sp.Rational(1, 25) * sp.cos(K1 + 1) * sp.cos(3 * PY)
    return phi_n, phi_1


def _vel_general():
    """(u^n, v^n, u^{n-1}, v^{n-1}): zero on both walls, not divergence-free."""
    s1, s2 = sp.sin(PY), sp.sin(2 * PY)
    u_n = sp.cos(K1) * s1 + sp.Rational(3, 10) * sp.sin(2 * K1 + sp.Rational(1, 2)) * s2
    v_n = sp.Rational(2, 5) * sp.sin(K1 + sp.Rational(1, 5)) * s1 * s1 + sp.Rational(1, 5) * sp.cos(K1) * s2
    u_p = u_n + sp.Rational(3, 10) * sp.sin(K1 + 1) * s1
    v_p = v_n - sp.Rational(1, 4) * sp.cos(2 * K1) * s2
    return u_n, v_n, u_p, v_p


def _vel_solenoidal():
    """Divergence-free levels from stream functions psi = sin^2(pi y) f(x):
    u = psi_y, v = -psi_x, both zero on the walls."""
    def from_psi(psi):
        return sp.diff(psi, Y_), -sp.diff(psi, X_)
    s2 = sp.sin(PY) ** 2
    u_n, v_n = from_psi(s2 * (sp.cos(K1) + sp.Rational(1, 2) * sp.sin(2 * K1)))
    du, dv = from_psi(s2 * sp.sin(K1 + 1) + sp.Rational(1, 3) * sp.sin(2 * PY) ** 2 * sp.cos(K1))
    return u_n, v_n, u_n + sp.Rational(2, 5) * du, v_n + sp.Rational(2, 5) * dv


def _grad(f):
    return sp.diff(f, X_), sp.diff(f, Y_)


def _div(fx, fy):
    return sp.diff(fx, X_) + sp.diff(fy, Y_)


def _lap(f):
    return sp.diff(f, X_, 2) + sp.diff(f, Y_, 2)


def _exact_rhs(prm, phi_n, phi_1, u_n, v_n, u_p, v_p, terms):
    """The continuous right-hand side (without the body force) from the
    listed terms, evaluated later at the nodes."""
    rho = prm.rho_water
    eta_bar = max(prm.eta_water, prm.eta_biofilm)
    ph = (phi_n + phi_1) / 2
    us, vs = sp.Rational(3, 2) * u_n - u_p / 2, sp.Rational(3, 2) * v_n - v_p / 2
    bu = rho * u_n / prm.dt
    bv = rho * v_n / prm.dt
    if "convection" in terms:
        bu -= rho * (us * sp.diff(us, X_) + vs * sp.diff(us, Y_))
        bv -= rho * (us * sp.diff(vs, X_) + vs * sp.diff(vs, Y_))
    if "capillary" in terms:
        gx, gy = _grad(ph)
        bu -= prm.gamma_cap * _div(gx * gx, gx * gy)
        bv -= prm.gamma_cap * _div(gx * gy, gy * gy)
    if "viscous" in terms or "viscous_paper" in terms:
        bu += eta_bar / 2 * _lap(u_n)
        bv += eta_bar / 2 * _lap(v_n)
        ep = ph * prm.eta_biofilm + (1 - ph) * prm.eta_water - eta_bar
        if "viscous" in terms:
            ex, ey = _grad(ep)
            bu += _div(ep * sp.diff(us, X_), ep * sp.diff(us, Y_)) + ex * sp.diff(us, X_) + ey * sp.diff(vs, X_)
            bv += _div(ep * sp.diff(vs, X_), ep * sp.diff(vs, Y_)) + ex * sp.diff(us, Y_) + ey * sp.diff(vs, Y_)
        else:
            # div(2 eta' D(v)), D = (grad v + grad v^T)/2: the stress of Eq. 4.1
            dxx, dyy = sp.diff(us, X_), sp.diff(vs, Y_)
            dxy = (sp.diff(us, Y_) + sp.diff(vs, X_)) / 2
            bu += _div(2 * ep * dxx, 2 * ep * dxy)
            bv += _div(2 * ep * dxy, 2 * ep * dyy)
    return bu, bv


def _momentum_errors(Om, prm, levels, terms, ns=(32, 64, 128)):
    phi_n, phi_1, u_n, v_n, u_p, v_p = levels
    eu, ev = _exact_rhs(prm, phi_n, phi_1, u_n, v_n, u_p, v_p, terms)
    fun = {k: _num(e) for k, e in dict(phi_n=phi_n, phi_1=phi_1, u_n=u_n, v_n=v_n,
                                         u_p=u_p, v_p=v_p, eu=eu, ev=ev).items()}
    errs = []
    for n in ns:
        p = prm.replace(nx=n, ny=n)
        g = Om.grid_of(p)
        X, Y = _coords(g)
        val = {k: f(X, Y) for k, f in fun.items()}
        for k in ("u_n", "v_n", "u_p", "v_p"):    # exact zeros on the walls
            val[k][0] = 0.0
            val[k][-1] = 0.0
        st = Om.State(val["phi_n"], val["phi_n"], val["u_n"], val["u_p"], val["v_n"], val["v_p"],
                      np.zeros(g.shape), 0.0)
        bu, bv = Om.momentum_rhs(p, g, st, val["phi_1"])
        f = Om.body_force_x(p)
        err = max(np.max(np.abs(bu - f - val["eu"])[1:-1]), np.max(np.abs(bv - val["ev"])[1:-1]))
        scale = max(np.max(np.abs(val["eu"])), np.max(np.abs(val["ev"])))
        errs.append(err / scale)
    return errs


def _assert_order2(errs, lo=1.85, hi=2.2):
    r = _rate(errs)
    assert all(lo < x < hi for x in r), (errs, r)


def _prm(**kw):
    base = dict(lx=LX, ly=LY, dt=0.5, eta_water=1.0, eta_biofilm=10.0, rho_water=1.3,
                rho_biofilm=1.3, gamma_cap=0.35, flow_mode=I.FLOW_POISEUILLE, u_max=1.0)
    base.update(kw)
    return I.Params(**base)


# checks (each takes the oracle module, so a planted mistake can be re-run) --

def check_convection(Om):
    """rho (v* . grad) v* alone: Gamma = 0, eta_b = eta_w (so eta' = 0)."""
    phi_n, phi_1 = _phi_levels()
    prm = _prm(gamma_cap=0.0, eta_biofilm=1.0)
    _assert_order2(_momentum_errors(Om, prm, (phi_n, phi_1) + _vel_general(), ("convection", "viscous")))


def check_capillary(Om):
    """-Gamma div(grad phi (x) grad phi) at phi^{n+1/2}, with the fluid at rest
    and no body force (shear mode with a still top wall)."""
    phi_n, phi_1 = _phi_levels()
    prm = _prm(flow_mode=I.FLOW_SHEAR, u_max=0.0)
    z = sp.Integer(0)
    _assert_order2(_momentum_errors(Om, prm, (phi_n, phi_1, z, z, z, z), ("capillary",)))


def check_viscous(Om):
    """The viscous terms alone (rho = 0 removes u/dt and the convection;
    Gamma = 0): eta_bar/2 Lap u^n + div(eta' grad v*) + (grad v*)^T grad eta'
    with a general (compressible) velocity and non-constant eta'."""
    phi_n, phi_1 = _phi_levels()
    prm = _prm(rho_water=0.0, rho_biofilm=0.0, gamma_cap=0.0)
    _assert_order2(_momentum_errors(Om, prm, (phi_n, phi_1) + _vel_general(), ("viscous",)))


def check_viscous_paper_form(Om):
    """For a divergence-free v* the remainder is div(2 eta' D(v*)) (Eq. 4.1)."""
    phi_n, phi_1 = _phi_levels()
    prm = _prm(rho_water=0.0, rho_biofilm=0.0, gamma_cap=0.0)
    _assert_order2(_momentum_errors(Om, prm, (phi_n, phi_1) + _vel_solenoidal(), ("viscous_paper",)))


def check_full(Om):
    """Every term at once, body force and wall rows included."""
    phi_n, phi_1 = _phi_levels()
    prm = _prm()
    _assert_order2(_momentum_errors(Om, prm, (phi_n, phi_1) + _vel_general(),
                                    ("convection", "capillary", "viscous")))


def check_face_forms(Om):
    """d/dx(c df/dx) and d/dy(c df/dy) in their compact face-mean forms."""
    c = 1 + sp.Rational(2, 5) * sp.sin(K1 + sp.Rational(3, 10)) * sp.cos(PY) \
        + sp.Rational(1, 5) * sp.cos(2 * K1) * sp.sin(2 * PY)
    f = sp.cos(K1 + 1) * sp.sin(PY) + sp.Rational(1, 3) * sp.sin(2 * K1) * sp.cos(2 * PY)
    ex_, ey_ = _num(sp.diff(c * sp.diff(f, X_), X_)), _num(sp.diff(c * sp.diff(f, Y_), Y_))
    fc, ff = _num(c), _num(f)
    e1, e2 = [], []
    for n in (32, 64, 128):
        g = O.Grid(n, n, LX, LY)
        X, Y = _coords(g)
        C, F = fc(X, Y), ff(X, Y)
        e1.append(np.max(np.abs(Om.dxx_face(g, C, F) - ex_(X, Y))))
        e2.append(np.max(np.abs((Om.dyy_face(g, C, F) - ey_(X, Y))[1:-1])))
        assert np.all(Om.dyy_face(g, C, F)[[0, -1]] == 0.0)
    _assert_order2(e1)
    _assert_order2(e2)


def check_wall_rows(Om):
    """Wall rows carry rho/dt times the Dirichlet values: u = 0 / u_top in
    shear mode, v = 0 (Eq. 4.3)."""
    prm = _prm(flow_mode=I.FLOW_SHEAR, u_max=0.25, nx=16, ny=12)
    g = Om.grid_of(prm)
    rng = np.random.default_rng(5)
    f = lambda: 0.3 + 0.4 * rng.random(g.shape)
    st = Om.State(f(), f(), f(), f(), f(), f(), np.zeros(g.shape), 0.0)
    bu, bv = Om.momentum_rhs(prm, g, st, f())
    c0 = prm.rho_water / prm.dt
    assert np.all(bu[0] == 0.0) and np.allclose(bu[-1], c0 * 0.25, rtol=1e-15, atol=0)
    assert np.all(bv[0] == 0.0) and np.all(bv[-1] == 0.0)


CHECKS = [check_convection, check_capillary, check_viscous, check_viscous_paper_form,
          check_full, check_face_forms, check_wall_rows]


@pytest.mark.parametrize("check", CHECKS, ids=lambda c: c.__name__)
def test_momentum_pin(check):
    check(O)


# planted mistakes ------------------------------------------------------------

_ORIG_CAP = O.capillary_force
_ORIG_MOM = O.momentum_rhs


def _cap_sign(prm, g, ph):
    cx, cy = _ORIG_CAP(prm, g, ph)
    return -cx, -cy


def _visc_no_transpose(g, ep, us, vs):
    return (O.dxx_face(g, ep, us) + O.dyy_face(g, ep, us),
            O.dxx_face(g, ep, vs) + O.dyy_face(g, ep, vs))


def _visc_transposed_operand(g, ep, us, vs):
    ex, ey = O.dx_c(g, ep), O.dy_c(g, ep)
    return (O.dxx_face(g, ep, us) + O.dyy_face(g, ep, us) + ex * O.dx_c(g, us) + ey * O.dy_c(g, us),
            O.dxx_face(g, ep, vs) + O.dyy_face(g, ep, vs) + ex * O.dx_c(g, vs) + ey * O.dy_c(g, vs))


def _dxx_node(g, c, f):
    return c * (O.xp(f) - 2.0 * f + O.xm(f)) / g.hx ** 2


def _dyy_node(g, c, f):
    out = np.zeros_like(f)
    out[1:-1] = c[1:-1] * (f[2:] - 2.0 * f[1:-1] + f[:-2]) / g.hy ** 2
    return out


def _conv_swapped(g, us, vs):
    return (vs * O.dx_c(g, us) + us * O.dy_c(g, us),
            vs * O.dx_c(g, vs) + us * O.dy_c(g, vs))


def _conv_v_minus_u(g, us, vs):
    # the second advecting component taken from the wrong field in v's row
    return (us * O.dx_c(g, us) + vs * O.dy_c(g, us),
            us * O.dx_c(g, vs) + us * O.dy_c(g, vs))


def _mom_phi_new_level(prm, g, st, phi_new):
    # capillary and viscosity at phi^{n+1} instead of phi^{n+1/2}
    return _ORIG_MOM(prm, g, dataclasses.replace(st, phi=phi_new), phi_new)


MUTANTS = {
    "capillary_sign": ("capillary_force", _cap_sign),
    "dropped_transpose_term": ("viscous_remainder", _visc_no_transpose),
    "transposed_gradient": ("viscous_remainder", _visc_transposed_operand),
    "dxx_node_values": ("dxx_face", _dxx_node),
    "dyy_node_values": ("dyy_face", _dyy_node),
    "convection_u_v_swapped": ("convection", _conv_swapped),
    "convection_wrong_component": ("convection", _conv_v_minus_u),
    "phase_field_level": ("momentum_rhs", _mom_phi_new_level),
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
    assert failed, f"planted mistake {name} passed every momentum pin"


def test_identity_patch_passes(monkeypatch):
    """The patching itself breaks nothing: the unchanged functions re-set pass."""
    for attr in ("capillary_force", "viscous_remainder", "convection", "dxx_face", "dyy_face"):
        monkeypatch.setattr(O, attr, getattr(O, attr))
    for check in CHECKS:
        check(O)
