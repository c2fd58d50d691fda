"""Pins of the oracle's nutrient transport and network production
(Eq. 2.5-2.7) against closed forms that do not come from the oracle.

Both wall conditions are pinned.  Zero total flux on both walls (the
boundary block of §2, the default): exact eigenvectors of the evenly
reflected second difference (cos(pi m j / ny)), the uniform consumption
decay, and the nutrient budget identity sum_W (phi_s c)^{n+1} - (phi_s c)^n
= -dt A/2 sum_W phi^{n+1/2} (c^{n+1} + c^n) on a state with flow.  c =
c_bulk on the top wall (nutrient_bc = 1): eigenvectors with a Dirichlet
row above (cos((2m+1) pi j / (2 ny))), the exact discrete steady boundary
layer (c_b cosh(beta j) / cosh(beta ny)), Couette advection of a Fourier
mode and the pointwise production step.  A dropped 1/2, a wrong time level
of phi_s, a sign or a wall treatment changes one of them at O(1).
"""
import dataclasses
import math

import numpy as np
import pytest

from oracle import cahn_oracle as O
from paper_1811_11842_gb300 import inputs


def _prm(**kw):
    """c = c_bulk on the top wall (nutrient_bc = 1)."""
    base = dict(nx=16, ny=12, lx=2.0, ly=1.0, mobility=0.0, u_max=0.0, dt=1e-2,
                nutrient=1, growth_mu=0.0, consume_a=40.0, diff_s=0.7, c_bulk=0.0,
                nutrient_bc=O.NUT_BC_BULK_TOP)
    base.update(kw)
    return inputs.Params(**base)


def _prm_flux(**kw):
    """Zero total flux on both walls (the default, nutrient_bc = 0)."""
    return _prm(nutrient_bc=O.NUT_BC_ZERO_FLUX, **kw)


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


# --------------------------------------------------------------------------
# zero total flux on both walls (the default)

@pytest.mark.parametrize("k,m", [(1, 0), (2, 3), (0, 12), (5, 1)])
def test_zero_flux_eigenmode_decays_by_the_crank_nicolson_factor(k, m):
    """Uniform phi, no flow: cos(2 pi k i/nx) cos(pi m j/ny) is an
    eigenvector of the evenly reflected diffusion on every row (walls
    included), eigenvalue 4/hx^2 sin^2(pi k/nx) + 4/hy^2 sin^2(pi m/(2 ny))."""
    prm = _prm_flux()
    phi0 = 0.3
    phi, u, v, p = _uniform(prm, phi0)
    i, j = _coords(prm)
    c0 = np.cos(2 * math.pi * k * i / prm.nx) * np.cos(math.pi * m * j / prm.ny) + 0.0 * phi
    hx, hy = prm.lx / prm.nx, prm.ly / prm.ny
    lam = (4 / hx ** 2 * math.sin(math.pi * k / prm.nx) ** 2
           + 4 / hy ** 2 * math.sin(math.pi * m / (2 * prm.ny)) ** 2)
    ps = 1.0 - phi0
    a = prm.consume_a
    rho = ((ps / prm.dt - 0.5 * a * phi0 - 0.5 * prm.diff_s * ps * lam)
           / (ps / prm.dt + 0.5 * a * phi0 + 0.5 * prm.diff_s * ps * lam))
    st = O.run(prm, phi, u, v, p, 3, c0=c0)
    np.testing.assert_allclose(st.c, rho ** 3 * c0, rtol=0, atol=1e-12)


def test_zero_flux_production_and_uniform_consumption():
    """Uniform phi and c, no flow: every node follows the pointwise steps
    phi^1 = phi^0 + dt g_n and (ps^1/dt + A ph/2) c^1 = (ps^0/dt - A ph/2) c^0,
    walls included; the mass target follows <phi, 1>_W."""
    prm = _prm_flux(growth_mu=3.0, growth_kc=0.15, growth_eps=0.5, consume_a=25.0,
                    c_bulk=0.9, dt=2e-2, mobility=1e-3)
    phi0 = 0.35
    phi, u, v, p = _uniform(prm, phi0)
    c0 = np.full_like(phi, 0.8)
    g = O.grid_of(prm)
    st1 = O.run(prm, phi, u, v, p, 1, c0=c0)
    phi1 = phi0 + prm.dt * prm.growth_eps * prm.growth_mu * phi0 * 0.8 / (prm.growth_kc + 0.8)
    np.testing.assert_allclose(st1.phi, phi1, rtol=1e-13)
    ph = 0.5 * (phi1 + phi0)
    a = prm.consume_a
    c1 = 0.8 * ((1 - phi0) / prm.dt - 0.5 * a * ph) / ((1 - phi1) / prm.dt + 0.5 * a * ph)
    np.testing.assert_allclose(st1.c, c1, rtol=1e-13)
    assert abs(st1.m0 - O.mass(g, st1.phi)) <= 1e-13 * st1.m0


@pytest.mark.parametrize("steps", [1, 3])
def test_zero_flux_nutrient_budget(steps):
    """On a state with protrusions, Poiseuille flow and a random c: every
    flux of Eq. 2.6 is a divergence with zero wall flux, so each step obeys
    sum_W (phi_s c)^{n+1} - sum_W (phi_s c)^n = -dt A/2 sum_W phi^{n+1/2}
    (c^{n+1} + c^n), to the solver tolerance."""
    prm = _prm_flux(nx=24, ny=16, mobility=1e-3, u_max=0.8, dt=1e-3, consume_a=30.0,
                    diff_s=0.4, growth_mu=0.5, eps=0.08)
    geo = inputs.Protrusions(h_b=0.25, centres=(1.0,), radius=0.2, noise=1e-3, seed=2)
    phi, u, v, p = inputs.initial_state(prm, geo)
    c0 = 0.4 + 0.5 * inputs.random_field(prm, 8, 0.0, 1.0)
    g = O.grid_of(prm)
    st = O.init_state(prm, phi, u, v, p, c0)
    for _ in range(steps):
        new = O.step(prm, st)
        ph = 0.5 * (new.phi + st.phi)
        lhs = O.mass(g, (1 - new.phi) * new.c) - O.mass(g, (1 - st.phi) * st.c)
        rhs = -prm.dt * 0.5 * prm.consume_a * O.mass(g, ph * (new.c + st.c))
        scale = O.mass(g, (1 - st.phi) * st.c)
        assert abs(lhs - rhs) <= 1e-12 * scale, (lhs, rhs)
        assert abs(rhs) > 1e-4 * scale          # consumption is active
        st = new


def test_zero_flux_operator_is_w_symmetric_positive():
    prm = _prm_flux(nx=6, ny=6)
    g = O.grid_of(prm)
    phi_new = 0.1 + 0.8 * inputs.random_field(prm, 3, 0.0, 1.0)
    phi_old = 0.1 + 0.8 * inputs.random_field(prm, 4, 0.0, 1.0)
    K = O.assemble(lambda x: O.nut_apply(prm, g, phi_new, phi_old, x), g.shape)
    S = np.diag(g.w.ravel()) @ K
    np.testing.assert_allclose(S, S.T, rtol=0, atol=1e-10 * np.abs(S).max())
    assert np.linalg.eigvalsh(0.5 * (S + S.T)).min() > 0


def test_zero_flux_cg_solution_matches_dense_lu():
    prm = _prm_flux(nx=8, ny=8)
    g = O.grid_of(prm)
    phi_new = 0.1 + 0.8 * inputs.random_field(prm, 5, 0.0, 1.0)
    phi_old = 0.1 + 0.8 * inputs.random_field(prm, 6, 0.0, 1.0)
    b = inputs.random_field(prm, 7)
    x_lu, _ = O.solve_nut(prm, g, phi_new, phi_old, b, method="lu")
    x_cg, its = O.solve_nut(prm, g, phi_new, phi_old, b)
    assert its > 0
    np.testing.assert_allclose(x_cg, x_lu, rtol=0, atol=1e-11 * np.abs(x_lu).max())


def test_couette_advection_uses_the_extrapolated_levels():
    """D = A = 0, Couette flow u = U y/Ly, uniform phi shifted by delta on
    step 1 (through the mass target), c^0 = cos(kx).  With sigma =
    sin(k hx)/hx, D_x cos = -sigma sin and D_x sin = sigma cos:
      step 1 (phi* = phi^0, c* = c^0):
        ps^1 c^1 = ps^0 c^0 + dt u ps^0 sigma sin(kx);
      step 2 (phi^2 = phi^1, phi* = phi^0 + 3 delta/2, c* = (3c^1 - c^0)/2):
        ps^1 c^2 = ps^1 c^1 - dt u ps* D_x c*."""
    prm = _prm_flux(diff_s=0.0, consume_a=0.0, flow_mode=O.FLOW_SHEAR, u_max=0.7)
    phi0, delta = 0.25, 0.04
    phi, u, v, p = _uniform(prm, phi0)
    i, j = _coords(prm)
    hx = prm.lx / prm.nx
    kx = 2 * math.pi * 3 / prm.lx
    x = i * hx
    cos, sin = np.cos(kx * x) + 0.0 * j, np.sin(kx * x) + 0.0 * j
    g = O.grid_of(prm)
    st = O.init_state(prm, phi, u, v, p, cos.copy())
    st.m0 = O.mass(g, phi) + delta * float(np.sum(g.w))
    st1 = O.step(prm, st)
    st2 = O.step(prm, st1)
    U = prm.u_max * (j * prm.ly / prm.ny) / prm.ly + 0.0 * i
    sig = math.sin(kx * hx) / hx
    ps0, ps1 = 1 - phi0, 1 - phi0 - delta
    alpha, beta = ps0 / ps1, prm.dt * U * ps0 * sig / ps1
    c1 = alpha * cos + beta * sin
    np.testing.assert_allclose(st1.phi, phi0 + delta, rtol=1e-14)
    np.testing.assert_allclose(st1.c, c1, rtol=0, atol=1e-12)
    pss = 1 - (phi0 + 1.5 * delta)
    dxcs = -(1.5 * alpha - 0.5) * sig * sin + 1.5 * beta * sig * cos
    c2 = c1 - prm.dt * U * pss * dxcs / ps1
    np.testing.assert_allclose(st2.phi, phi0 + delta, rtol=1e-14)
    np.testing.assert_allclose(st2.c, c2, rtol=0, atol=1e-12)


# --------------------------------------------------------------------------
# Planted mistakes: each must make at least one of the pins above fail.  The
# mistake is planted in the oracle module for the duration of one test
# (monkeypatch restores it).

def _pins():
    return [
        lambda: test_eigenmode_decays_by_the_crank_nicolson_factor(1, 0),
        test_discrete_steady_state_is_a_fixed_point,
        test_couette_advection_of_a_fourier_mode,
        test_production_and_time_levels_of_the_solid_fraction,
        test_production_clamps_a_negative_extrapolated_nutrient,
        test_operator_is_w_symmetric_positive_on_the_dirichlet_free_space,
        test_diffusion_coefficient_is_taken_at_the_half_level,
        lambda: test_zero_flux_eigenmode_decays_by_the_crank_nicolson_factor(2, 3),
        test_zero_flux_production_and_uniform_consumption,
        lambda: test_zero_flux_nutrient_budget(1),
        test_zero_flux_operator_is_w_symmetric_positive,
        test_couette_advection_uses_the_extrapolated_levels,
    ]


_orig_coeff = O.nut_coefficients
_orig_apply = O.nut_apply
_orig_growth = O.growth


def _coeff_diag_old(prm, phi_new, phi_old):
    diag, ks, ph = _orig_coeff(prm, phi_new, phi_old)
    return diag + (phi_new - phi_old) / prm.dt, ks, ph          # phi_s^n in the diagonal


def _coeff_k_new(prm, phi_new, phi_old):
    diag, _, ph = _orig_coeff(prm, phi_new, phi_old)
    return diag, prm.diff_s * (1.0 - phi_new), ph                # k at phi^{n+1}


def _coeff_a_full(prm, phi_new, phi_old):
    diag, ks, ph = _orig_coeff(prm, phi_new, phi_old)
    return diag + 0.5 * prm.consume_a * ph, ks, ph               # A instead of A/2


def _apply_no_half(prm, g, phi_new, phi_old, x):
    diag, ks, _ = _orig_coeff(prm, phi_new, phi_old)
    y = diag * x + O.ga(g, ks, x)                                # G_k instead of G_k / 2
    if O.nut_dirichlet_top(prm):
        y[-1] = x[-1] / prm.dt
    return y


def _growth_no_saturation(prm, phis, cs):
    return prm.growth_eps * prm.growth_mu * phis * np.maximum(cs, 0.0)   # K_c dropped


MUTANTS = {
    "diagonal at phi_s^n": ("nut_coefficients", _coeff_diag_old),
    "diffusion coefficient at phi^{n+1}": ("nut_coefficients", _coeff_k_new),
    "consumption without 1/2": ("nut_coefficients", _coeff_a_full),
    "diffusion without 1/2": ("nut_apply", _apply_no_half),
    "production without saturation": ("growth", _growth_no_saturation),
    "top wall always Dirichlet": ("nut_dirichlet_top", lambda prm: True),
    "top wall never Dirichlet": ("nut_dirichlet_top", lambda prm: False),
    "no extrapolation": ("extrapolate", lambda q, q_prev: q.copy()),
}


@pytest.mark.parametrize("name", list(MUTANTS))
def test_planted_mistake_is_caught(monkeypatch, name):
    attr, bad = MUTANTS[name]
    monkeypatch.setattr(O, attr, bad)
    failed = []
    for pin in _pins():
        try:
            pin()
        except Exception as e:          # a broken oracle may fail any way
            failed.append(type(e).__name__)
    assert failed, f"planted mistake not caught: {name}"


def _near_one_state(prm):
    """phi just below 1 everywhere (phi* stays inside (0, 1)), fluid at rest."""
    g = O.grid_of(prm)
    rng = np.random.default_rng(7)
    phi = 0.9995 + 1e-5 * rng.random(g.shape)
    z = np.zeros(g.shape)
    return phi, z, z.copy(), z.copy(), np.ones(g.shape)


def test_nutrient_domain_error_when_phi_reaches_one():
    """The nutrient lives in phi_s = 1 - phi (Eq. 2.6): a mass target that
    the correction can only reach with phi^{n+1} > 1 stops the step before
    the nutrient solve; the same state with a reachable target steps."""
    prm = inputs.config_nutrient()[0].replace(nx=16, ny=12, eps=0.2, dt=1e-4)
    g = O.grid_of(prm)
    st = O.init_state(prm, *_near_one_state(prm))
    sw = float(np.sum(g.w))
    ok = O.step(prm, dataclasses.replace(st, m0=st.m0 + 2e-4 * sw))
    assert np.all(ok.phi < 1.0)
    with pytest.raises(O.DomainError):
        O.step(prm, dataclasses.replace(st, m0=st.m0 + 2e-3 * sw))
