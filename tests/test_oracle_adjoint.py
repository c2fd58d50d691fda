"""Pins of the oracle's discrete adjoint: a dot-product test of every
transposed operator (<A x, y> = <x, A^T y> for random x, y), and the full
gradient against central finite differences of the forward oracle."""
import numpy as np
import pytest

from oracle import cahn_adjoint as A
from oracle import cahn_oracle as O
from paper_1811_11842_gb300 import inputs as I


def _g(nx=16, ny=12):
    return O.Grid(nx, ny, 2.0, 1.0)


def _dot_test(fwd, bwd, shape_in, shape_out, seed=0, tol=1e-12):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(shape_in)
    y = rng.standard_normal(shape_out)
    lhs = np.sum(fwd(x) * y)
    rhs = np.sum(x * bwd(y))
    assert abs(lhs - rhs) <= tol * max(abs(lhs), 1.0), (lhs, rhs)


def test_transposes_of_difference_operators():
    g = _g()
    sh = g.shape
    _dot_test(lambda x: O.dx_c(g, x), lambda y: A.dx_c_T(g, y), sh, sh)
    _dot_test(lambda x: O.dy_c(g, x), lambda y: A.dy_c_T(g, y), sh, sh)
    _dot_test(lambda x: O.div_c(g, x, 0 * x), lambda y: A.div_c_T(g, y)[0], sh, sh)
    _dot_test(lambda x: O.div_c(g, 0 * x, x), lambda y: A.div_c_T(g, y)[1], sh, sh)
    _dot_test(lambda x: O.lap(g, x), lambda y: A.lap_T(g, y), sh, sh)
    _dot_test(lambda x: O.even_rows(x)[2:], A.north_T, sh, sh)
    _dot_test(lambda x: O.even_rows(x)[:-2], A.south_T, sh, sh)


def test_transposes_of_variable_coefficient_operators():
    g = _g()
    sh = g.shape
    rng = np.random.default_rng(4)
    a = 0.3 + rng.random(sh)
    z = rng.standard_normal(sh)
    _dot_test(lambda x: O.ga(g, a, x), lambda y: A.ga_T(g, a, y), sh, sh)
    _dot_test(lambda c: O.ga(g, c, z), lambda y: A.ga_coef_T(g, z, y), sh, sh)
    c0 = 0.5 + rng.random(sh)
    f0 = rng.standard_normal(sh)
    _dot_test(lambda f: O.dxx_face(g, c0, f), lambda y: A.dxx_face_T(g, c0, f0, y)[1], sh, sh)
    _dot_test(lambda c: O.dxx_face(g, c, f0), lambda y: A.dxx_face_T(g, c0, f0, y)[0], sh, sh)
    _dot_test(lambda f: O.dyy_face(g, c0, f), lambda y: A.dyy_face_T(g, c0, f0, y)[1], sh, sh)
    _dot_test(lambda c: O.dyy_face(g, c, f0), lambda y: A.dyy_face_T(g, c0, f0, y)[0], sh, sh)


def _small_problem(nx=16, ny=16):
    prm, geo, _ = I.config_small()
    prm = prm.replace(nx=nx, ny=ny, eps=0.08, dt=2e-4, mobility=5e-3, u_max=1.0)
    geo = I.Protrusions(h_b=0.3, centres=(1.0,), radius=0.2, noise=1e-3, seed=1)
    return prm, I.initial_state(prm, geo)


def test_momentum_rhs_transpose():
    prm, (phi, u, v, p) = _small_problem()
    g = O.grid_of(prm)
    rng = np.random.default_rng(8)
    st = O.init_state(prm, phi, u + 0.01 * rng.standard_normal(u.shape), v + 0.01 * rng.standard_normal(v.shape), p)
    st.u_prev = st.u - 0.01 * rng.standard_normal(u.shape)
    st.v_prev = st.v - 0.01 * rng.standard_normal(v.shape)
    phi_new = phi + 0.01 * rng.standard_normal(phi.shape)
    us, vs = O.extrapolate(st.u, st.u_prev), O.extrapolate(st.v, st.v_prev)
    bu_b, bv_b = rng.standard_normal(phi.shape), rng.standard_normal(phi.shape)
    bars = A.momentum_rhs_T(prm, g, st, phi_new, us, vs, bu_b, bv_b)
    names = ["phi_new", "phi", "us", "vs", "u", "v"]
    dirs = {k: rng.standard_normal(phi.shape) for k in names}

    def rhs(eps):
        s2 = st.copy()
        pn = phi_new + eps * dirs["phi_new"]
        s2.phi = st.phi + eps * dirs["phi"]
        # us = 1.5 u - 0.5 u_prev; perturb us through u_prev, u through u with us fixed
        s2.u = st.u + eps * dirs["u"]
        s2.u_prev = st.u_prev + eps * (3.0 * dirs["u"] - 2.0 * dirs["us"])
        s2.v = st.v + eps * dirs["v"]
        s2.v_prev = st.v_prev + eps * (3.0 * dirs["v"] - 2.0 * dirs["vs"])
        bu, bv = O.momentum_rhs(prm, g, s2, pn)
        bu[0] = bu[-1] = bv[0] = bv[-1] = 0.0
        return np.sum(bu * bu_b) + np.sum(bv * bv_b)

    h = 1e-6
    fd = (rhs(h) - rhs(-h)) / (2 * h)
    ad = sum(np.sum(b * dirs[k]) for k, b in zip(names, bars))
    assert abs(fd - ad) <= 1e-7 * max(abs(fd), 1.0), (fd, ad)


def _fd_gradient(prm, state, nsteps, d_phi0):
    def J(prm_, phi0):
        st = O.run(prm_, phi0, *state[1:], nsteps, rtol=1e-15)
        return A.objective(prm_, st.phi)
    out = {}
    for name in ("chi", "mobility"):
        v = getattr(prm, name)
        h = 1e-6 * abs(v)
        out[name] = (J(prm.replace(**{name: v + h}), state[0])
                     - J(prm.replace(**{name: v - h}), state[0])) / (2 * h)
    h = 1e-6
    out["phi0"] = (J(prm, state[0] + h * d_phi0) - J(prm, state[0] - h * d_phi0)) / (2 * h)
    return out


def test_gradient_matches_central_differences():
    prm, state = _small_problem()
    nsteps = 4
    Jv, phi0_b, chi_b, mob_b = A.gradient(prm, *state, nsteps)
    d = I.random_field(prm, seed=31)
    d /= np.sqrt(np.mean(d * d))                 # unit-RMS direction
    fd = _fd_gradient(prm, state, nsteps, d)
    for name, ad in (("chi", chi_b), ("mobility", mob_b), ("phi0", float(np.sum(phi0_b * d)))):
        assert abs(ad - fd[name]) <= 1e-5 * abs(fd[name]), (name, ad, fd[name])


def test_gradient_double_well_shear():
    prm, state = _small_problem(nx=12, ny=10)
    prm = prm.replace(energy=O.ENERGY_DOUBLE_WELL, gamma2=2.0, stab_s=1.0,
                      flow_mode=O.FLOW_SHEAR, u_max=0.5)
    state = I.initial_state(prm, I.Protrusions(h_b=0.3, centres=(1.0,), radius=0.2, seed=2))
    Jv, phi0_b, chi_b, mob_b = A.gradient(prm, *state, 3)
    d = I.random_field(prm, seed=5)
    fd = _fd_gradient(prm, state, 3, d)
    assert abs(mob_b - fd["mobility"]) <= 1e-5 * abs(fd["mobility"])
    assert abs(np.sum(phi0_b * d) - fd["phi0"]) <= 1e-5 * abs(fd["phi0"])
