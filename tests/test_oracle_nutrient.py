"""Pins of the oracle's nutrient transport and network production
(Eq. 2.5-2.7) against closed forms that do not come from the oracle.

The discrete operators are pinned through exact eigenvectors of the
second difference with a zero-flux row below and a Dirichlet row above
(cos((2m+1) pi j / (2 ny))), the exact discrete steady state
(c_b cosh(beta j) / cosh(beta ny)), the central difference of a Fourier
mode under a Couette flow, and the pointwise production ODE step.  A
dropped 1/2, a wrong time level of phi_s, a sign or a wall treatment
changes one of them at O(1).
"""
import math

import numpy as np
import pytest

from oracle import cahn_oracle as O
from paper_1811_11842_gb300 import inputs


def _prm(**kw):
    base = dict(nx=16, ny=12, lx=2.0, ly=1.0, mobility=0.0, u_max=0.0, dt=1e-2,
                nutrient=1, growth_mu=0.0, consume_a=40.0, diff_s=0.7, c_bulk=0.0)
    base.update(kw)
    return inputs.Params(**base)


def _uniform(prm, phi0):
    phi = np.full((prm.ny + 1, prm.nx), phi0)
    u, v, p = inputs.initial_velocity(prm)
    return phi, u, v, p


def _coords(prm):
    i = np.arange(prm.nx)[None, :]
    j = np.arange(prm.ny + 1)[:, None]
    return i, j


@pytest.mark.parametrize("k,m", [(1, 0), (3, 2), (0, 5)])
def test_eigenmode_decays_by_the_crank_nicolson_factor(k, m):
    """Uniform phi, no flow, c_bulk = 0: cos(2 pi k i/nx) cos(theta j) with
    theta = (2m+1) pi / (2 ny) is an eigenvector of the zero-flux/Dirichlet
    diffusion, so each step multiplies it by
    (ps/dt - A phi/2 - D ps lam/2) / (ps/dt + A phi/2 + D ps lam/2)."""
    prm = _prm()
    phi0 = 0.3
    phi, u, v, p = _uniform(prm, phi0)
    i, j = _coords(prm)
    th = (2 * m + 1) * math.pi / (2 * prm.ny)
    c0 = np.cos(2 * math.pi * k * i / prm.nx) * np.cos(th * j) + 0.0 * phi
    hx, hy = prm.lx / prm.nx, prm.ly / prm.ny
    lam = 4 / hx ** 2 * math.sin(math.pi * k / prm.nx) ** 2 + 4 / hy ** 2 * math.sin(th / 2) ** 2
    ps = 1.0 - phi0
    num = ps / prm.dt - 0.5 * prm.consume_a * phi0 - 0.5 * prm.diff_s * ps * lam
    den = ps / prm.dt + 0.5 * prm.consume_a * phi0 + 0.5 * prm.diff_s * ps * lam
    rho = num / den
    st = O.run(prm, phi, u, v, p, 3, c0=c0)
    np.testing.assert_allclose(st.c, rho ** 3 * c0, rtol=0, atol=1e-12)
    np.testing.assert_allclose(st.phi, phi, rtol=0, atol=1e-14)


def test_discrete_steady_state_is_a_fixed_point():
    """Uniform phi, no flow, c = c_b cosh(beta j)/cosh(beta ny) with
    cosh(beta) = 1 + A phi hy^2 / (2 D ps): consumption balances diffusion
    on every row below the wall and the wall holds c_b, so a step returns
    the same field."""
    prm = _prm(c_bulk=0.8, consume_a=300.0)
    phi0 = 0.4
    phi, u, v, p = _uniform(prm, phi0)
    i, j = _coords(prm)
    hy = prm.ly / prm.ny
    ps = 1.0 - phi0
    beta = math.acosh(1.0 + prm.consume_a * phi0 * hy ** 2 / (2 * prm.diff_s * ps))
    c0 = prm.c_bulk * np.cosh(beta * j) / math.cosh(beta * prm.ny) + 0.0 * i
    assert c0[0, 0] < 0.5 * prm.c_bulk   # a real boundary layer
    st = O.run(prm, phi, u, v, p, 2, c0=c0)
    np.testing.assert_allclose(st.c, c0, rtol=1e-12, atol=0)


def test_couette_advection_of_a_fourier_mode():
    """D = A = 0, uniform phi, u = U y / Ly (the Couette profile the shear
    flow keeps): c^1 = c^0 - dt u D_x c^0 with the central difference
    D_x cos(kx) = -sin(kx) sin(k hx) / hx (phi_s cancels)."""
    prm = _prm(diff_s=0.0, consume_a=0.0, flow_mode=O.FLOW_SHEAR, u_max=0.7, c_bulk=0.3)
    phi, u, v, p = _uniform(prm, 0.25)
    i, j = _coords(prm)
    kx = 2 * math.pi * 2 / prm.lx
    hx = prm.lx / prm.nx
    x = i * hx
    c0 = np.cos(kx * x) + 0.0 * j
    st = O.run(prm, phi, u, v, p, 1, c0=c0)
    y = j * (prm.ly / prm.ny)
    want = c0 + prm.dt * (prm.u_max * y / prm.ly) * np.sin(kx * x) * math.sin(kx * hx) / hx
    np.testing.assert_allclose(st.c[:-1], want[:-1], rtol=0, atol=1e-12)
    np.testing.assert_allclose(st.c[-1], prm.c_bulk, rtol=0, atol=0)
    np.testing.assert_allclose(st.u, u, rtol=0, atol=1e-12)


def test_production_and_time_levels_of_the_solid_fraction():
    """M = 0 and D = 0 decouple the nodes.  Step 1: phi^1 = phi^0 + dt eps mu
    phi^0 c^0 / (K_c + c^0) and (ps^1/dt + A ph/2) c^1 = (ps^0/dt - A ph/2)
    c^0 with ph = (phi^1 + phi^0)/2.  Step 2 uses the extrapolated phi*, c*.
    The mass target follows <phi, 1>_W exactly."""
    prm = _prm(diff_s=0.0, growth_mu=3.0, growth_kc=0.15, growth_eps=0.5, consume_a=25.0,
               c_bulk=0.9, dt=2e-2)
    phi0 = 0.35
    phi, u, v, p = _uniform(prm, phi0)
    c0 = np.full_like(phi, prm.c_bulk)
    g = O.grid_of(prm)
    gfun = lambda ph, c: prm.growth_eps * prm.growth_mu * ph * c / (prm.growth_kc + c)
    st1 = O.run(prm, phi, u, v, p, 1, c0=c0)
    phi1 = phi0 + prm.dt * gfun(phi0, prm.c_bulk)
    np.testing.assert_allclose(st1.phi, phi1, rtol=1e-13)
    ph = 0.5 * (phi1 + phi0)
    a = prm.consume_a
    c1 = prm.c_bulk * ((1 - phi0) / prm.dt - 0.5 * a * ph) / ((1 - phi1) / prm.dt + 0.5 * a * ph)
    np.testing.assert_allclose(st1.c[:-1], c1, rtol=1e-13)
    np.testing.assert_allclose(st1.c[-1], prm.c_bulk, rtol=0, atol=0)
    assert abs(st1.m0 - O.mass(g, st1.phi)) <= 1e-13 * st1.m0
    # step 2: phi* = (3 phi^1 - phi^0)/2, c* likewise (top row: c_bulk)
    st2 = O.step(prm, st1)
    phis = 1.5 * phi1 - 0.5 * phi0
    cs = 1.5 * c1 - 0.5 * prm.c_bulk
    want = np.full_like(phi, phi1 + prm.dt * gfun(phis, cs))
    want[-1] = phi1 + prm.dt * gfun(phis, prm.c_bulk)
    np.testing.assert_allclose(st2.phi, want, rtol=1e-13)
    assert abs(st2.m0 - O.mass(g, st2.phi)) <= 1e-13 * st2.m0


def test_production_clamps_a_negative_extrapolated_nutrient():
    """g_n uses max(c*, 0): an extrapolated c* < 0 produces nothing."""
    prm = _prm()
    phis = np.array([0.3, 0.3])
    cs = np.array([-0.5, 0.5])
    gn = O.growth(prm.replace(growth_mu=1.0), phis, cs)
    assert gn[0] == 0.0 and gn[1] > 0.0


def test_operator_is_w_symmetric_positive_on_the_dirichlet_free_space():
    """K restricted to fields with a zero top row is symmetric and positive
    definite in <.,.>_W (the property that lets CG solve it)."""
    prm = _prm(nx=6, ny=6)
    g = O.grid_of(prm)
    phi_new = 0.1 + 0.8 * inputs.random_field(prm, 3, 0.0, 1.0)
    phi_old = 0.1 + 0.8 * inputs.random_field(prm, 4, 0.0, 1.0)
    K = O.assemble(lambda x: O.nut_apply(prm, g, phi_new, phi_old, x), g.shape)
    nf = prm.nx * prm.ny                     # rows 0..ny-1
    W = np.diag(g.w.ravel()[:nf])
    S = W @ K[:nf, :nf]
    np.testing.assert_allclose(S, S.T, rtol=0, atol=1e-10 * np.abs(S).max())
    assert np.linalg.eigvalsh(0.5 * (S + S.T)).min() > 0
    # the top row is the decoupled Dirichlet row
    top = K[nf:, :]
    np.testing.assert_allclose(top[:, nf:], np.eye(prm.nx) / prm.dt, rtol=0, atol=0)
    assert not np.any(top[:, :nf])


def test_cg_solution_matches_dense_lu():
    prm = _prm(nx=8, ny=8, c_bulk=0.6)
    g = O.grid_of(prm)
    phi_new = 0.1 + 0.8 * inputs.random_field(prm, 5, 0.0, 1.0)
    phi_old = 0.1 + 0.8 * inputs.random_field(prm, 6, 0.0, 1.0)
    b = inputs.random_field(prm, 7)
    b[-1] = prm.c_bulk / prm.dt
    x_lu, _ = O.solve_nut(prm, g, phi_new, phi_old, b, method="lu")
    x_cg, its = O.solve_nut(prm, g, phi_new, phi_old, b)
    assert its > 0
    np.testing.assert_allclose(x_cg, x_lu, rtol=0, atol=1e-11 * np.abs(x_lu).max())
    np.testing.assert_allclose(x_lu[-1], prm.c_bulk, rtol=1e-14)


def test_diffusion_coefficient_is_taken_at_the_half_level():
    """A mass target above <phi^0, 1>_W shifts phi uniformly (M = 0, no
    production): phi^1 = phi^0 + delta.  The eigenmode of the first test
    then decays by (ps^0/dt - D ps^h lam/2) / (ps^1/dt + D ps^h lam/2)
    with ps^h = 1 - (phi^0 + phi^1)/2 (A = 0)."""
    prm = _prm(consume_a=0.0, diff_s=1.3)
    phi0, delta = 0.3, 0.05
    phi, u, v, p = _uniform(prm, phi0)
    i, j = _coords(prm)
    th = 3 * math.pi / (2 * prm.ny)
    c0 = np.cos(2 * math.pi * 2 * i / prm.nx) * np.cos(th * j) + 0.0 * phi
    g = O.grid_of(prm)
    st = O.init_state(prm, phi, u, v, p, c0)
    st.m0 = O.mass(g, phi) + delta * float(np.sum(g.w))
    st1 = O.step(prm, st)
    np.testing.assert_allclose(st1.phi, phi0 + delta, rtol=1e-14)
    hx, hy = prm.lx / prm.nx, prm.ly / prm.ny
    lam = 4 / hx ** 2 * math.sin(math.pi * 2 / prm.nx) ** 2 + 4 / hy ** 2 * math.sin(th / 2) ** 2
    psh = 1.0 - (phi0 + 0.5 * delta)
    rho = (((1 - phi0) / prm.dt - 0.5 * prm.diff_s * psh * lam)
           / ((1 - phi0 - delta) / prm.dt + 0.5 * prm.diff_s * psh * lam))
    np.testing.assert_allclose(st1.c, rho * c0, rtol=0, atol=1e-12)
