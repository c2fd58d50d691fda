"""FP64 discrete adjoint of the oracle's time step (McClanahan et al. §4).

TEST INFRASTRUCTURE ONLY.  Gives the exact gradient of an objective of the
final phase field, J(phi^N), with respect to the initial phase field phi^0,
the Flory-Huggins chi and the mobility M, through N steps of
`cahn_oracle.step`.  Every step is differentiated exactly: each elementary
operation of the forward code is reversed here (transposes in the
Euclidean inner product of the flattened arrays), and the three linear
solves are reversed by solving with the transposed matrices (dense, so
this is for small grids).  Pinned by dot-product tests of every transpose
and by central finite differences of the forward oracle.

Objective used by the workloads: the detached-biofilm volume
J = sum over rows with y_j > 0.25 of w_ij phi_ij dx dy (rows at exactly
0.25 excluded).
"""
from __future__ import annotations

import numpy as np

from . import cahn_oracle as O


# --------------------------------------------------------------------------
# transposes of the elementary operators

def xp_T(lam):      # transpose of x_{i+1} (roll -1) is roll +1
    return O.xm(lam)


def xm_T(lam):
    return O.xp(lam)


def dx_c_T(g, lam):
    """Central periodic derivative is antisymmetric."""
    return -O.dx_c(g, lam)


def dy_c_T(g, lam):
    """Transpose of dy_c (output on interior rows only)."""
    out = np.zeros_like(lam)
    t = lam[1:-1] / (2.0 * g.hy)
    out[2:] += t
    out[:-2] -= t
    return out


def dy_odd_T(g, lam):
    """Transpose of the y part of div_c (flux odd-reflected at the walls)."""
    out = np.zeros_like(lam)
    t = lam[1:-1] / (2.0 * g.hy)
    out[2:] += t
    out[:-2] -= t
    out[1] += lam[0] / g.hy
    out[-2] -= lam[-1] / g.hy
    return out


def div_c_T(g, lam):
    return dx_c_T(g, lam), dy_odd_T(g, lam)


def north_T(lam):
    """Transpose of a -> even_rows(a)[2:] (north neighbour, reflected)."""
    out = np.zeros_like(lam)
    out[1:] += lam[:-1]
    out[-2] += lam[-1]
    return out


def south_T(lam):
    """Transpose of a -> even_rows(a)[:-2] (south neighbour, reflected)."""
    out = np.zeros_like(lam)
    out[:-1] += lam[1:]
    out[1] += lam[0]
    return out


def lap_T(g, lam):
    """L_h is W-symmetric: L^T = W L W^-1."""
    return g.w * O.lap(g, lam / g.w)


def ga_T(g, a, lam):
    """G_a is W-symmetric: G_a^T = W G_a W^-1."""
    return g.w * O.ga(g, a, lam / g.w)


def ga_coef_T(g, z, lam):
    """Transpose of the map a -> G_a z (linear in a) applied to lam."""
    ze = O.even_rows(z)
    dze = O.xp(z) - z
    dzw = z - O.xm(z)
    dzn = ze[2:] - z
    dzs = z - ze[:-2]
    ae_b = -lam * dze / g.hx ** 2
    aw_b = lam * dzw / g.hx ** 2
    an_b = -lam * dzn / g.hy ** 2
    as_b = lam * dzs / g.hy ** 2
    a_b = 0.5 * (ae_b + xp_T(ae_b)) + 0.5 * (aw_b + xm_T(aw_b))
    a_b += 0.5 * (an_b + north_T(an_b)) + 0.5 * (as_b + south_T(as_b))
    return a_b


def dxx_face_T(g, c, f, lam):
    """(c_bar, f_bar) of dxx_face(c, f) against lam."""
    t = lam / g.hx ** 2
    ce = 0.5 * (c + O.xp(c))
    cw = 0.5 * (c + O.xm(c))
    f_b = xp_T(ce * t) - ce * t - cw * t + xm_T(cw * t)
    ce_b = t * (O.xp(f) - f)
    cw_b = -t * (f - O.xm(f))
    c_b = 0.5 * (ce_b + xp_T(ce_b)) + 0.5 * (cw_b + xm_T(cw_b))
    return c_b, f_b


def dyy_face_T(g, c, f, lam):
    """(c_bar, f_bar) of dyy_face(c, f) (interior rows) against lam."""
    t = lam[1:-1] / g.hy ** 2
    cn = 0.5 * (c[1:-1] + c[2:])
    cs = 0.5 * (c[1:-1] + c[:-2])
    f_b = np.zeros_like(f)
    f_b[2:] += cn * t
    f_b[1:-1] -= cn * t + cs * t
    f_b[:-2] += cs * t
    cn_b = t * (f[2:] - f[1:-1])
    cs_b = -t * (f[1:-1] - f[:-2])
    c_b = np.zeros_like(c)
    c_b[1:-1] += 0.5 * (cn_b + cs_b)
    c_b[2:] += 0.5 * cn_b
    c_b[:-2] += 0.5 * cs_b
    return c_b, f_b


def lap_int_T(g, lam):
    """Transpose of the interior-row Laplacian with stored wall neighbours."""
    t = np.zeros_like(lam)
    t[1:-1] = lam[1:-1]
    out = np.zeros_like(lam)
    c = t[1:-1]
    # x part: (2c - xm(c) - xp(c)) / hx^2 is symmetric in the periodic direction
    out[1:-1] += (2.0 * c - O.xm(c) - O.xp(c)) / g.hx ** 2
    # y part: 2 f_j - f_{j-1} - f_{j+1}
    out[1:-1] += 2.0 * c / g.hy ** 2
    out[:-2] -= c / g.hy ** 2
    out[2:] -= c / g.hy ** 2
    return out


def f_second(prm, phi):
    if prm.energy == O.ENERGY_DOUBLE_WELL:
        return 2.0 * prm.gamma2 * (1.0 - 6.0 * phi + 6.0 * phi * phi)
    return 1.0 / (prm.n_poly * phi) + 1.0 / (1.0 - phi) - 2.0 * prm.chi


def f_prime_dchi(prm, phi):
    if prm.energy == O.ENERGY_DOUBLE_WELL:
        return np.zeros_like(phi)
    return 1.0 - 2.0 * phi


# --------------------------------------------------------------------------
# dense transposed solves (small grids)

class DenseSolves:
    """Dense matrices of H and of the bordered pressure system (constant),
    and of A_phi for a given coefficient (assembled per step)."""

    def __init__(self, prm, g):
        self.prm, self.g = prm, g
        n = g.shape[0] * g.shape[1]
        self.n = n
        self.H = O.assemble(lambda x: O.helm_apply(prm, g, x), g.shape)
        Lm = O.assemble(lambda x: O.lap(g, x), g.shape)
        M = np.zeros((n + 1, n + 1))
        M[:n, :n] = Lm
        M[:n, n] = 1.0
        M[n, :n] = g.w.ravel()
        self.Mp = M

    def a_phi(self, a):
        return O.assemble(lambda x: O.ch_apply(self.prm, self.g, a, x), self.g.shape)

    def helm_T(self, ybar):
        """b_bar of x = H^-1 b, with the wall rows of b fixed (constants)."""
        bb = np.linalg.solve(self.H.T, ybar.ravel()).reshape(self.g.shape)
        bb[0] = 0.0
        bb[-1] = 0.0
        return bb

    def poisson_T(self, pbar):
        """d_bar of p = poisson_solve(d) (projection, bordered solve)."""
        g = self.g
        n = self.n
        rhs = np.concatenate([pbar.ravel(), [0.0]])
        z = np.linalg.solve(self.Mp.T, rhs)[:n].reshape(g.shape)
        # d -> d - <d,1>_W / <1,1>_W has transpose y -> y - w (1^T y) / sum(w)
        return z - g.w * np.sum(z) / np.sum(g.w)


# --------------------------------------------------------------------------
# one step forward with a tape, and its reverse

def step_tape(prm, st):
    g = O.grid_of(prm)
    rho = O.rho0(prm)
    a, phis = O.ch_coefficient(prm, st)
    us = O.extrapolate(st.u, st.u_prev)
    vs = O.extrapolate(st.v, st.v_prev)
    psi_n = prm.kappa * O.lap(g, st.phi) + prm.stab_s * st.phi
    w = 0.5 * psi_n + O.f_prime(prm, phis) - prm.stab_s * phis
    b = O.ch_rhs(prm, g, st)[0]
    phit, _ = O.solve_phi(prm, g, a, b, x0=st.phi, rtol=1e-15)
    phi_new = phit + (st.m0 - O.mass(g, phit)) / float(np.sum(g.w))
    bu, bv = O.momentum_rhs(prm, g, st, phi_new)
    ut = O.helm_solve(prm, g, bu)
    vt = O.helm_solve(prm, g, bv)
    d = rho * O.div_c(g, ut, vt)
    p = O.poisson_solve(prm, g, d)
    px, py = O.grad_c(g, p)
    u_new, v_new = ut.copy(), vt.copy()
    u_new[1:-1] += px[1:-1] / rho
    v_new[1:-1] += py[1:-1] / rho
    new = O.State(phi_new, st.phi, u_new, st.u, v_new, st.v, p, st.m0, st.step + 1)
    tape = dict(st=st, a=a, phis=phis, us=us, vs=vs, w=w, phit=phit, phi_new=phi_new)
    return new, tape


def momentum_rhs_T(prm, g, st, phi_new, us, vs, bu_b, bv_b):
    """Reverse of cahn_oracle.momentum_rhs: returns bars of (phi_new, phi^n,
    u*, v*, u^n, v^n) for the interior-row bars bu_b, bv_b."""
    rho = O.rho0(prm)
    nu = 0.5 * O.eta_bar(prm)
    gam = prm.gamma_cap
    bu_b = bu_b.copy()
    bv_b = bv_b.copy()
    bu_b[0] = bu_b[-1] = 0.0
    bv_b[0] = bv_b[-1] = 0.0
    ph = 0.5 * (phi_new + st.phi)
    eta = ph * prm.eta_biofilm + (1.0 - ph) * prm.eta_water
    ep = eta - O.eta_bar(prm)
    gx, gy = O.dx_c(g, ph), O.dy_c(g, ph)
    ex, ey = O.dx_c(g, ep), O.dy_c(g, ep)
    us_b = np.zeros_like(us)
    vs_b = np.zeros_like(vs)
    ep_b = np.zeros_like(ep)
    # rho u/dt and -nu lap_int(u)
    u_b = rho / prm.dt * bu_b - nu * lap_int_T(g, bu_b)
    v_b = rho / prm.dt * bv_b - nu * lap_int_T(g, bv_b)
    # convection -rho (us dx(us) + vs dy(us)),  -rho (us dx(vs) + vs dy(vs))
    cu = -rho * bu_b
    cv = -rho * bv_b
    us_b += cu * O.dx_c(g, us) + dx_c_T(g, us * cu) + dy_c_T(g, vs * cu)
    vs_b += cu * O.dy_c(g, us)
    us_b += cv * O.dx_c(g, vs)
    vs_b += dx_c_T(g, us * cv) + cv * O.dy_c(g, vs) + dy_c_T(g, vs * cv)
    # capillary -Gamma (dx(gx^2) + dy(gx gy)),  -Gamma (dx(gx gy) + dy(gy^2))
    t1 = -gam * dx_c_T(g, bu_b)
    t2 = -gam * dy_c_T(g, bu_b)
    t3 = -gam * dx_c_T(g, bv_b)
    t4 = -gam * dy_c_T(g, bv_b)
    gx_b = 2.0 * gx * t1 + gy * t2 + gy * t3
    gy_b = gx * t2 + gx * t3 + 2.0 * gy * t4
    ph_b = dx_c_T(g, gx_b) + dy_c_T(g, gy_b)
    # viscous remainder (x component)
    c_b, f_b = dxx_face_T(g, ep, us, bu_b)
    ep_b += c_b
    us_b += f_b
    c_b, f_b = dyy_face_T(g, ep, us, bu_b)
    ep_b += c_b
    us_b += f_b
    ex_b = bu_b * O.dx_c(g, us)
    us_b += dx_c_T(g, ex * bu_b)
    ey_b = bu_b * O.dx_c(g, vs)
    vs_b += dx_c_T(g, ey * bu_b)
    # viscous remainder (y component)
    c_b, f_b = dxx_face_T(g, ep, vs, bv_b)
    ep_b += c_b
    vs_b += f_b
    c_b, f_b = dyy_face_T(g, ep, vs, bv_b)
    ep_b += c_b
    vs_b += f_b
    ex_b += bv_b * O.dy_c(g, us)
    us_b += dy_c_T(g, ex * bv_b)
    ey_b += bv_b * O.dy_c(g, vs)
    vs_b += dy_c_T(g, ey * bv_b)
    ep_b += dx_c_T(g, ex_b) + dy_c_T(g, ey_b)
    ph_b += (prm.eta_biofilm - prm.eta_water) * ep_b
    return 0.5 * ph_b, 0.5 * ph_b, us_b, vs_b, u_b, v_b


def step_reverse(prm, tape, dense, phi_new_b, u_new_b, v_new_b):
    """Bars of (phi^n, phi^{n-1}, u^n, u^{n-1}, v^n, v^{n-1}), chi, M, m0 from
    the bars of (phi^{n+1}, u^{n+1}, v^{n+1})."""
    g = O.grid_of(prm)
    rho = O.rho0(prm)
    st = tape["st"]
    a, phis, us, vs, w = tape["a"], tape["phis"], tape["us"], tape["vs"], tape["w"]
    phit, phi_new = tape["phit"], tape["phi_new"]
    # 8. correction
    ut_b = u_new_b.copy()
    vt_b = v_new_b.copy()
    px_b = np.zeros_like(u_new_b)
    py_b = np.zeros_like(v_new_b)
    px_b[1:-1] = u_new_b[1:-1] / rho
    py_b[1:-1] = v_new_b[1:-1] / rho
    p_b = dx_c_T(g, px_b) + dy_c_T(g, py_b)
    # 7. pressure
    d_b = dense.poisson_T(p_b)
    fx_b, fy_b = div_c_T(g, rho * d_b)
    ut_b += fx_b
    vt_b += fy_b
    # 6. predictor solves
    bu_b = dense.helm_T(ut_b)
    bv_b = dense.helm_T(vt_b)
    # 5. momentum rhs
    pnew_b_m, phi_b, us_b, vs_b, u_b, v_b = momentum_rhs_T(prm, g, st, phi_new, us, vs, bu_b, bv_b)
    pn_b = phi_new_b + pnew_b_m
    # 3. mass correction
    s = np.sum(pn_b) / float(np.sum(g.w))
    phit_b = pn_b - g.w * s
    m0_b = s
    # 2. phase-field solve
    A = dense.a_phi(a)
    b_b = np.linalg.solve(A.T, phit_b.ravel()).reshape(g.shape)
    psi_t = prm.kappa * O.lap(g, phit) + prm.stab_s * phit
    a_b = -0.5 * ga_coef_T(g, psi_t, b_b)
    # 1. rhs b = phi^n/dt - G_a w - D_c(phi* u*, phi* v*)
    phi_b = phi_b + b_b / prm.dt
    w_b = -ga_T(g, a, b_b)
    a_b += -ga_coef_T(g, w, b_b)
    fx_b, fy_b = div_c_T(g, -b_b)
    phis_b = us * fx_b + vs * fy_b
    us_b = us_b + phis * fx_b
    vs_b = vs_b + phis * fy_b
    phi_b += 0.5 * (prm.kappa * lap_T(g, w_b) + prm.stab_s * w_b)
    phis_b += (f_second(prm, phis) - prm.stab_s) * w_b
    chi_b = float(np.sum(f_prime_dchi(prm, phis) * w_b))
    phis_b += prm.mobility * a_b
    mob_b = float(np.sum(phis * a_b))
    # extrapolations
    out = dict(phi=phi_b + 1.5 * phis_b, phi_prev=-0.5 * phis_b,
               u=u_b + 1.5 * us_b, u_prev=-0.5 * us_b,
               v=v_b + 1.5 * vs_b, v_prev=-0.5 * vs_b,
               chi=chi_b, mobility=mob_b, m0=m0_b)
    return out


def objective_weights(prm, y_cut=0.25):
    """dJ/dphi^N of the detached-volume objective (rows with y > y_cut)."""
    g = O.grid_of(prm)
    y = np.arange(prm.ny + 1) * g.hy
    mask = (y > y_cut).astype(np.float64)[:, None] * np.ones((1, prm.nx))
    return mask * g.w * g.hx * g.hy


def objective(prm, phi, y_cut=0.25):
    return float(np.sum(objective_weights(prm, y_cut) * phi))


def gradient(prm, phi0, u0, v0, p0, nsteps, jbar=None):
    """(J, dJ/dphi0, dJ/dchi, dJ/dM) through nsteps oracle steps."""
    g = O.grid_of(prm)
    st = O.init_state(prm, phi0, u0, v0, p0)
    tapes = []
    for _ in range(nsteps):
        st, tp = step_tape(prm, st)
        tapes.append(tp)
    if jbar is None:
        jbar = objective_weights(prm)
    J = float(np.sum(jbar * st.phi))
    dense = DenseSolves(prm, g)
    z = np.zeros(g.shape)
    bars = {nsteps: [jbar.copy(), z.copy(), z.copy()], nsteps - 1: [z.copy(), z.copy(), z.copy()]}
    chi_b = mob_b = m0_b = 0.0
    for n in range(nsteps - 1, -1, -1):
        pb, ub, vb = bars.pop(n + 1)
        r = step_reverse(prm, tapes[n], dense, pb, ub, vb)
        cur = bars.setdefault(n, [z.copy(), z.copy(), z.copy()])
        prv = bars.setdefault(n - 1, [z.copy(), z.copy(), z.copy()])
        cur[0] += r["phi"]
        cur[1] += r["u"]
        cur[2] += r["v"]
        prv[0] += r["phi_prev"]
        prv[1] += r["u_prev"]
        prv[2] += r["v_prev"]
        chi_b += r["chi"]
        mob_b += r["mobility"]
        m0_b += r["m0"]
    # phi^{-1} = phi^0 and m0 = <phi^0, 1>_W
    phi0_b = bars[0][0] + bars[-1][0] + g.w * m0_b
    return J, phi0_b, chi_b, mob_b
