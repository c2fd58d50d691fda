"""Pins of the FP64 oracle to facts that do not come from the oracle itself:
the paper's printed stencil (Listing 3), closed-form eigenpairs, library
dense solves and FFTs, complex-step derivatives, manufactured solutions
(second-order rates, §4 "second order accuracy") and conservation /
invariance properties of the scheme.  CPU only.

Each check is a function of the oracle module so that the planted-mistake
tests at the bottom can re-run it against a deliberately broken copy."""
import math
import os
import types

import numpy as np
import pytest
import sympy as sp

from oracle import cahn_oracle as O
from paper_1811_11842_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _grid(nx, ny, lx=2.0, ly=1.0):
    return O.Grid(nx, ny, lx, ly)


def _coords(g):
    x = np.arange(g.nx) * g.hx
    y = np.arange(g.ny + 1) * g.hy
    return np.meshgrid(x, y)


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# --------------------------------------------------------------------------
# Listing 3: the 5-point row 4, -1, -1, -1, -1 and the periodic wrap

def check_listing3(Om):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "listing3_laplacian_row.txt"))
            if l.strip() and not l.startswith("#")]
    vals = [float(v) for v in rows[0]]
    nx, ny = 8, 8
    g = Om.Grid(nx, ny, float(nx), float(ny))          # unit mesh widths
    A = Om.assemble(lambda x: Om.lap(g, x), g.shape)
    idx = lambda i, j: j * nx + (i % nx)
    for (i, j) in [(3, 4), (0, 4)]:                     # interior, and i-1 wraps
        r = idx(i, j)
        cols = [idx(i, j), idx(i - 1, j), idx(i + 1, j), idx(i, j - 1), idx(i, j + 1)]
        for c, v in zip(cols, vals):
            assert A[r, c] == v, (i, j, c, A[r, c], v)
        others = np.delete(A[r], cols)
        assert np.all(others == 0.0)
    assert rows[1][0] == "wrap" and A[idx(0, 4), idx(nx - 1, 4)] == -1.0


def test_listing3_row():
    check_listing3(O)


# --------------------------------------------------------------------------
# Closed-form eigenpairs (cos in x, cos / sin in y)

def check_lap_eigen(Om):
    g = _grid(24, 16)
    X, Y = _coords(g)
    for k, l in [(1, 0), (0, 1), (3, 5), (12, 16), (7, 9)]:
        v = np.cos(2 * np.pi * k * X / g.lx) * np.cos(np.pi * l * Y / g.ly)
        lam = 4 / g.hx ** 2 * math.sin(math.pi * k / g.nx) ** 2 \
            + 4 / g.hy ** 2 * math.sin(math.pi * l / (2 * g.ny)) ** 2
        assert _rel(Om.lap(g, v), lam * v) < 1e-12, (k, l)


def test_lap_eigen():
    check_lap_eigen(O)


def check_helm_eigen(Om):
    prm = I.Params(nx=24, ny=16, lx=2.0, ly=1.0, dt=1e-3, eta_water=1.0, eta_biofilm=4.0)
    g = Om.grid_of(prm)
    X, Y = _coords(g)
    c0, nu = 1.0 / prm.dt, 0.5 * 4.0
    for k, l in [(0, 1), (2, 3), (11, 15)]:
        v = np.cos(2 * np.pi * k * X / g.lx) * np.sin(np.pi * l * Y / g.ly)
        v[0] = v[-1] = 0.0
        lam = 4 / g.hx ** 2 * math.sin(math.pi * k / g.nx) ** 2 \
            + 4 / g.hy ** 2 * math.sin(math.pi * l / (2 * g.ny)) ** 2
        assert _rel(Om.helm_apply(prm, g, v), (c0 + nu * lam) * v) < 1e-12


def test_helm_eigen():
    check_helm_eigen(O)


def check_ch_const_eigen(Om):
    prm = I.Params(nx=16, ny=12, lx=2.0, ly=1.0, eps=0.05, dt=1e-3, stab_s=2.0)
    g = Om.grid_of(prm)
    X, Y = _coords(g)
    a = 0.7
    for k, l in [(1, 1), (5, 7), (8, 12)]:
        v = np.cos(2 * np.pi * k * X / g.lx) * np.cos(np.pi * l * Y / g.ly)
        lam = 4 / g.hx ** 2 * math.sin(math.pi * k / g.nx) ** 2 \
            + 4 / g.hy ** 2 * math.sin(math.pi * l / (2 * g.ny)) ** 2
        want = (1 / prm.dt + 0.5 * a * lam * (prm.kappa * lam + prm.stab_s)) * v
        got = Om.ch_apply(prm, g, a * np.ones(g.shape), v)
        assert _rel(got, want) < 1e-12


def test_ch_const_eigen():
    check_ch_const_eigen(O)


# --------------------------------------------------------------------------
# Variable coefficient operator: symmetry, conservation, positivity

def check_ga_structure(Om):
    g = _grid(20, 14)
    rng = np.random.default_rng(3)
    a = 0.2 + rng.random(g.shape)
    x, y = rng.standard_normal(g.shape), rng.standard_normal(g.shape)
    gx, gy = Om.ga(g, a, x), Om.ga(g, a, y)
    w = g.w
    assert abs(np.sum(w * gx * y) - np.sum(w * x * gy)) < 1e-11 * np.sum(np.abs(w * gx * y))
    assert abs(np.sum(w * gx)) < 1e-10 * np.sum(np.abs(gx))
    assert np.sum(w * gx * x) > 0
    # constant coefficient reduces to the scaled Laplacian
    assert _rel(Om.ga(g, 1.7 * np.ones(g.shape), x), 1.7 * Om.lap(g, x)) < 1e-13


def test_ga_structure():
    check_ga_structure(O)


# --------------------------------------------------------------------------
# Manufactured solutions: observed order 2 (§4)

_xs, _ys = sp.symbols("x y")


def _mms_fields(lx, ly):
    u = sp.cos(2 * sp.pi * _xs / lx) * sp.cos(sp.pi * _ys / ly) \
        + sp.Rational(3, 10) * sp.cos(4 * sp.pi * _xs / lx + 1) * sp.cos(2 * sp.pi * _ys / ly)
    a = 1 + sp.Rational(2, 5) * sp.sin(2 * sp.pi * _xs / lx + sp.Rational(3, 10)) \
        * sp.cos(sp.pi * _ys / ly)
    return u, a


def _num(expr):
    f = sp.lambdify((_xs, _ys), expr, "numpy")
    return lambda X, Y: np.broadcast_to(f(X, Y), X.shape).astype(np.float64)


def _rate(errs):
    return [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


def check_mms_ga(Om):
    lx, ly = 2.0, 1.0
    u, a = _mms_fields(lx, ly)
    exact = -(sp.diff(a * sp.diff(u, _xs), _xs) + sp.diff(a * sp.diff(u, _ys), _ys))
    fu, fa, fe = _num(u), _num(a), _num(exact)
    errs = []
    for n in (16, 32, 64):
        g = _grid(n, n, lx, ly)
        X, Y = _coords(g)
        errs.append(np.max(np.abs(Om.ga(g, fa(X, Y), fu(X, Y)) - fe(X, Y))))
    assert all(1.9 < r < 2.1 for r in _rate(errs)), errs


def test_mms_ga():
    check_mms_ga(O)


def check_mms_fourth_order(Om):
    """G_a L_h against -div(a grad(-Laplacian u)) for the fourth-order part."""
    lx, ly = 2.0, 1.0
    u, a = _mms_fields(lx, ly)
    lapu = -(sp.diff(u, _xs, 2) + sp.diff(u, _ys, 2))
    exact = -(sp.diff(a * sp.diff(lapu, _xs), _xs) + sp.diff(a * sp.diff(lapu, _ys), _ys))
    fu, fa, fe = _num(u), _num(a), _num(exact)
    errs = []
    for n in (32, 64, 128):
        g = _grid(n, n, lx, ly)
        X, Y = _coords(g)
        got = Om.ga(g, fa(X, Y), Om.lap(g, fu(X, Y)))
        errs.append(np.max(np.abs(got - fe(X, Y))) / np.max(np.abs(fe(X, Y))))
    assert all(1.85 < r < 2.15 for r in _rate(errs)), errs


def test_mms_fourth_order():
    check_mms_fourth_order(O)


def check_mms_div_grad(Om):
    lx, ly = 2.0, 1.0
    fx = sp.sin(2 * sp.pi * _xs / lx) * sp.cos(sp.pi * _ys / ly)
    fy = sp.cos(2 * sp.pi * _xs / lx) * sp.sin(sp.pi * _ys / ly)   # 0 on the walls
    p, _ = _mms_fields(lx, ly)
    dexact = sp.diff(fx, _xs) + sp.diff(fy, _ys)
    gxe, gye = sp.diff(p, _xs), sp.diff(p, _ys)
    e1, e2 = [], []
    for n in (16, 32, 64):
        g = _grid(n, n, lx, ly)
        X, Y = _coords(g)
        d = Om.div_c(g, _num(fx)(X, Y), _num(fy)(X, Y))
        e1.append(np.max(np.abs(d - _num(dexact)(X, Y))))
        gx, gy = Om.grad_c(g, _num(p)(X, Y))
        e2.append(max(np.max(np.abs(gx - _num(gxe)(X, Y))),
                      np.max(np.abs((gy - _num(gye)(X, Y))[1:-1]))))
        # exact discrete conservation: sum_W D_c F = 0 when F_y = 0 on walls
        assert abs(np.sum(g.w * d)) < 1e-11 * np.sum(np.abs(d))
    assert all(1.9 < r < 2.1 for r in _rate(e1)), e1
    assert all(1.9 < r < 2.1 for r in _rate(e2)), e2


def test_mms_div_grad():
    check_mms_div_grad(O)


def test_projection_divergence_rate():
    """After the projection (Eq. 4.4-4.5) the collocated central divergence
    of v is O(h^2) (compact L_h is not D_c grad_c)."""
    lx, ly = 2.0, 1.0
    prm0 = I.Params(lx=lx, ly=ly)
    ratios = []
    for n in (32, 64, 128):
        prm = prm0.replace(nx=n, ny=n)
        g = O.grid_of(prm)
        X, Y = _coords(g)
        u = np.sin(2 * np.pi * X / lx) * np.sin(np.pi * Y / ly) ** 2 + Y * (1 - Y)
        v = np.cos(2 * np.pi * X / lx) * np.sin(np.pi * Y / ly)
        p = O.poisson_solve(prm, g, O.div_c(g, u, v))
        px, py = O.grad_c(g, p)
        u2, v2 = u.copy(), v.copy()
        u2[1:-1] += px[1:-1]
        v2[1:-1] += py[1:-1]
        ratios.append(np.max(np.abs(O.div_c(g, u2, v2)[1:-1])))
    r = _rate(ratios)
    assert all(1.8 < x < 2.3 for x in r), ratios


# --------------------------------------------------------------------------
# Free energy: complex-step derivative, binodal, spinodal

def check_energy(Om):
    for energy, chi, g2 in [(O.ENERGY_FLORY_HUGGINS, 2.5, 0.0), (O.ENERGY_FLORY_HUGGINS, 2.9, 0.0),
                            (O.ENERGY_DOUBLE_WELL, 0.0, 3.0)]:
        prm = I.Params(chi=chi, energy=energy, gamma2=g2, n_poly=1.0)
        phi = np.linspace(0.05, 0.95, 37)
        h = 1e-30
        cs = np.imag(Om.f_bulk(prm, phi + 1j * h)) / h      # complex-step F'
        assert np.max(np.abs(Om.f_prime(prm, phi) - cs)) < 1e-12
    prm = I.Params(chi=2.5, n_poly=1.0)
    p_in, p_out = I.binodal_pair(2.5, 1.0)
    # symmetric binodal: common tangent of slope 0, equal bulk energies
    assert abs(Om.f_prime(prm, p_in)) < 1e-12 and abs(Om.f_prime(prm, p_out)) < 1e-12
    assert abs(Om.f_bulk(prm, p_in) - Om.f_bulk(prm, p_out)) < 1e-14
    # spinodal of N = 1: phi (1 - phi) = 1 / (2 chi), where F'' = 0
    ps = 0.5 * (1 + math.sqrt(1 - 2 / 2.5))
    fpp = np.imag(Om.f_prime(prm, ps + 1e-30j)) / 1e-30
    assert abs(fpp) < 1e-12


def test_energy_functions():
    check_energy(O)


# --------------------------------------------------------------------------
# Solvers against library dense LU and FFT

def _small(prm_kw=None):
    prm = I.Params(nx=16, ny=16, lx=2.0, ly=1.0, eps=0.05, dt=1e-3, mobility=0.5,
                   stab_s=0.5)
    if prm_kw:
        prm = prm.replace(**prm_kw)
    return prm, O.grid_of(prm)


def check_solvers_vs_dense(Om):
    prm, g = _small()
    rng = np.random.default_rng(7)
    a = 0.1 + rng.random(g.shape)
    b = rng.standard_normal(g.shape)
    ap = lambda x: Om.ch_apply(prm, g, a, x)
    ref = np.linalg.solve(Om.assemble(ap, g.shape), b.ravel()).reshape(g.shape)
    x, _ = Om.gmres(g, ap, b, rtol=1e-14, diag=Om.probe_diagonal(ap, g.shape))
    assert _rel(x, ref) < 1e-12
    # Helmholtz predictor: CG, FFT/DST and dense agree
    bh = rng.standard_normal(g.shape)
    hp = lambda x: Om.helm_apply(prm, g, x)
    refh = np.linalg.solve(Om.assemble(hp, g.shape), bh.ravel()).reshape(g.shape)
    assert _rel(Om.helm_solve(prm, g, bh), refh) < 1e-12
    xh, _ = Om.cg(g, hp, bh, rtol=1e-15)
    assert _rel(xh, refh) < 1e-12
    # singular pressure: bordered dense, FFT/DCT and projected CG agree
    d = rng.standard_normal(g.shape)
    refp = Om.dense_poisson_solve(g, d)
    assert abs(np.sum(g.w * refp)) < 1e-12
    assert _rel(Om.poisson_solve(prm, g, d), refp) < 1e-12
    dproj = d - np.sum(g.w * d) / np.sum(g.w)
    xp_, _ = Om.cg(g, lambda x: Om.lap(g, x), dproj, rtol=1e-15, project=True)
    assert _rel(xp_, refp) < 1e-11
    # constant-coefficient CH: spectral vs dense
    ac = 0.3
    apc = lambda x: Om.ch_apply(prm, g, ac * np.ones(g.shape), x)
    refc = np.linalg.solve(Om.assemble(apc, g.shape), b.ravel()).reshape(g.shape)
    assert _rel(Om.ch_const_solve(prm, g, ac, b), refc) < 1e-12


def test_solvers_vs_dense():
    check_solvers_vs_dense(O)


def test_probe_diagonal_matches_dense():
    prm, g = _small()
    a = 0.1 + np.random.default_rng(1).random(g.shape)
    ap = lambda x: O.ch_apply(prm, g, a, x)
    A = O.assemble(ap, g.shape)
    assert np.allclose(O.probe_diagonal(ap, g.shape).ravel(), np.diag(A), rtol=1e-14, atol=0)


# --------------------------------------------------------------------------
# Time step: invariants and special cases

def check_mass_conservation(Om, nsteps=20):
    """With zero-flux walls Eq. 2.4 conserves <phi,1>_W exactly; before the
    mass correction the drift is only the solver tolerance."""
    prm, geo, _ = I.config_small()
    g = Om.grid_of(prm)
    st = Om.init_state(prm, *I.initial_state(prm, geo))
    m0 = st.m0
    worst = 0.0
    for _ in range(nsteps):
        b, a, _ = Om.ch_rhs(prm, g, st)
        phi_new, _ = Om.solve_phi(prm, g, a, b, x0=st.phi)
        worst = max(worst, abs(Om.mass(g, phi_new) - Om.mass(g, st.phi)) / m0)
        st = Om.step(prm, st)
    assert worst <= 1e-12, worst


def test_mass_conservation():
    check_mass_conservation(O)


def test_energy_decay_no_flow():
    """No flow: the discrete free energy does not increase step to step."""
    prm, geo, _ = I.config_small()
    g = O.grid_of(prm)
    st = O.init_state(prm, *I.initial_state(prm, geo))
    e = [O.energy(prm, g, st.phi)]
    zero = np.zeros(g.shape)
    for _ in range(20):
        st.u = st.u_prev = st.v = st.v_prev = zero
        b, a, _ = O.ch_rhs(prm, g, st)
        phi_new, _ = O.solve_phi(prm, g, a, b, x0=st.phi)
        st.phi_prev, st.phi = st.phi, phi_new
        e.append(O.energy(prm, g, st.phi))
    d = np.diff(e)
    assert np.all(d <= 1e-12 * abs(e[0])), d


def test_constant_phi_invariant():
    prm = I.Params(nx=32, ny=16, u_max=0.0, dt=1e-3)
    g = O.grid_of(prm)
    phi = 0.3 * np.ones(g.shape)
    z = np.zeros(g.shape)
    st = O.run(prm, phi, z, z, z, 5)
    assert np.max(np.abs(st.phi - 0.3)) < 1e-13
    assert max(np.max(np.abs(st.u)), np.max(np.abs(st.v)), np.max(np.abs(st.p))) < 1e-12


def test_poiseuille_steady_state():
    """Uniform viscosity: the parabolic profile is an exact discrete steady
    state (quadratics are differenced exactly) with p = 0."""
    prm = I.Params(nx=32, ny=16, eta_water=2.0, eta_biofilm=2.0, u_max=1.0, dt=1e-3)
    u0, v0, p0 = I.initial_velocity(prm)
    phi = 0.4 * np.ones_like(u0)
    st = O.run(prm, phi, u0, v0, p0, 5)
    assert np.max(np.abs(st.u - u0)) < 1e-11
    assert np.max(np.abs(st.v)) < 1e-12 and np.max(np.abs(st.p)) < 1e-12


def test_y_only_phi_stays_x_independent():
    prm = I.Params(nx=32, ny=32, u_max=0.0, dt=1e-4)
    _, y = I.grid_coords(prm)
    phi = 0.5 + 0.3 * np.tanh((y[:, None] - 0.4) / 0.05) * np.ones((1, prm.nx))
    z = np.zeros_like(phi)
    st = O.run(prm, phi, z, z, z, 4)
    assert np.max(np.abs(st.phi - st.phi[:, :1])) < 1e-13
    assert np.max(np.abs(st.u)) < 1e-12


def test_domain_error():
    prm = I.Params(nx=16, ny=16)
    g = O.grid_of(prm)
    phi = 0.5 * np.ones(g.shape)
    phi[3, 3] = 1.2
    z = np.zeros(g.shape)
    with pytest.raises(O.DomainError):
        O.step(prm, O.init_state(prm, phi, z, z, z))


# --------------------------------------------------------------------------
# Planted mistakes: each must make at least one pin fail

def _mutant(**overrides):
    m = types.ModuleType("oracle_mutant")
    m.__dict__.update(O.__dict__)
    m.__dict__.update(overrides)
    return m


def test_mutant_face_coefficient_not_averaged():
    def ga_bad(g, a, x):
        xe = O.even_rows(x)
        fx = a * (O.xp(x) - x) - a * (x - O.xm(x))
        fy = a * (xe[2:] - x) - a * (x - xe[:-2])
        return -(fx / g.hx ** 2 + fy / g.hy ** 2)
    m = _mutant(ga=ga_bad)
    with pytest.raises(AssertionError):
        check_ga_structure(m)


def test_mutant_wall_reflection_odd():
    def lap_bad(g, x):
        e = O.odd_rows(x)
        s, c, n = e[:-2], e[1:-1], e[2:]
        return (2.0 * c - O.xm(c) - O.xp(c)) / g.hx ** 2 + (2.0 * c - s - n) / g.hy ** 2
    with pytest.raises(AssertionError):
        check_lap_eigen(_mutant(lap=lap_bad))


def test_mutant_x_y_mesh_swapped():
    def lap_bad(g, x):
        e = O.even_rows(x)
        s, c, n = e[:-2], e[1:-1], e[2:]
        return (2.0 * c - O.xm(c) - O.xp(c)) / g.hy ** 2 + (2.0 * c - s - n) / g.hx ** 2
    with pytest.raises(AssertionError):
        check_listing3(_mutant(lap=lap_bad)) if False else check_lap_eigen(_mutant(lap=lap_bad))


def test_mutant_dropped_half_in_cn():
    def ch_bad(prm, g, a, x):
        return x / prm.dt + O.ga(g, a, prm.kappa * O.lap(g, x) + prm.stab_s * x)
    with pytest.raises(AssertionError):
        check_ch_const_eigen(_mutant(ch_apply=ch_bad))


def test_mutant_fprime_sign():
    def fp_bad(prm, phi):
        return (np.log(phi) + 1.0) / prm.n_poly - np.log(1.0 - phi) - 1.0 - prm.chi * (1.0 - 2.0 * phi)
    with pytest.raises(AssertionError):
        check_energy(_mutant(f_prime=fp_bad))


def test_mutant_divergence_not_conservative():
    def div_bad(g, fx, fy):
        ye = O.even_rows(fy)
        return O.dx_c(g, fx) + (ye[2:] - ye[:-2]) / (2.0 * g.hy) + 0.0 * fy + fy * 1e-3
    with pytest.raises(AssertionError):
        check_mms_div_grad(_mutant(div_c=div_bad))
