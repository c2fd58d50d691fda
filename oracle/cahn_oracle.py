"""FP64 CPU oracle for the per-time-step linear solves of the modified
Cahn-Hilliard biofilm model coupled to incompressible flow by a projection
method (McClanahan, Stegmeier, Sundermann, Doom, Kimn, "Parallel Simulations
of Biofilm Flow using the Modified Cahn-Hilliard Equation", §2-§4).

TEST INFRASTRUCTURE ONLY.  This module exists to check the CUDA library.
Only the test suite, the smoke check and the CPU-baseline leg of the
benchmark may import it; the product path never does.  It shares no code
with the CUDA path: the one common import is the seeded input module.

Plain numpy, FP64 throughout, no blocking or fusion.  Each function cites
the passage it follows.  Readings of passages that are silent, garbled or
in conflict:

  * Grid (§4, nodes (i dx, j dy)): nx periodic columns, ny + 1 rows
    j = 0..ny, walls on rows 0 and ny.  Trapezoid weights w = 1/2 on wall
    rows, 1 elsewhere; every inner product below is <x, y>_W = sum(w x y).
  * Zero-flux walls (Eq. 4.6) are imposed by even reflection of ghost rows,
    two deep for the fourth-order operator (Eq. 4.7).
  * Face coefficients of the variable-coefficient operator are arithmetic
    means of the nodal values (the paper is silent).
  * Free energy: Flory-Huggins F(phi) = phi ln(phi)/N + (1-phi) ln(1-phi)
    + chi phi (1-phi) by default; the paper's double well
    Gamma2 phi^2 (1-phi)^2 (Eq. 2.3, 3.3) is kept as an option.
  * Time discretisation (§4, "Crank-Nicolson and extrapolation"):
    CN on the linear stiff terms, the n+1/2 extrapolation
    q* = (3 q^n - q^{n-1}) / 2 for the nonlinear ones; q^{-1} = q^0.
  * Momentum (Eq. 4.1-4.3, garbled there): CN on eta_bar Laplacian with
    eta_bar = max(eta_water, eta_biofilm); the rest of the variable
    viscous stress, the capillary force -Gamma div(grad phi grad phi)
    (the divergence lost in Eq. 3.3 restored from Eq. 2.2 and 4.1), the
    convection and the body force are explicit.  The explicit viscous
    remainder div(2 eta' D(v)), eta' = eta - eta_bar, is written in its
    divergence-free form div(eta' grad v) + (grad v)^T grad eta' -- the
    same identity Eq. 4.1-4.2 use to trade (2/Re_a) D for the Laplacian.
    (The full form's grad-div part has twice the coefficient and, on the
    collocated grid, acts on compressive modes the projection cannot see;
    with a 10:1 viscosity ratio it is unstable.)
  * Flow: POISEUILLE = no-slip on both walls, driven by the constant body
    force f_x = 8 eta_water u_max / Ly^2; SHEAR = the paper's top-wall
    speed (Eq. 5.2).
  * Pressure (Eq. 4.4): the singular Neumann problem is made compatible by
    the W-weighted projection d <- d - <d,1>_W / <1,1>_W (the weighted
    form of the paper's constant null-space removal, Listing 5), gauge
    <p, 1>_W = 0.  Sign as printed: v = u + grad(p)/rho (Eq. 4.5).
  * Mass correction after the phi solve restores <phi, 1>_W to its target:
    the initial value, advanced each step by dt <g_n, 1>_W when the
    network production g_n is on (changes phi by the solver tolerance
    only: every other term of Eq. 2.4 is a divergence).
  * Nutrient (Eq. 2.6-2.7, optional; the paper gives no time
    discretisation for it): unknown c on the same nodes, phi_s = 1 - phi.
    Crank-Nicolson on diffusion and consumption with the coefficients at
    phi^{n+1/2} = (phi^{n+1} + phi^n)/2, the time derivative
    (phi_s^{n+1} c^{n+1} - phi_s^n c^n)/dt, the advective flux c* phi_s* v*
    extrapolated like the phase field's.  Walls as in the boundary block of
    §2: zero total nutrient flux on y = 0 and y = Ly (the normal velocity
    vanishes there, so the advective flux is odd and c is evenly
    reflected); optionally (nutrient_bc = 1) c = c_bulk on the top wall
    instead.  The production g_n of Eq. 2.5 enters the phase-field rhs at
    the extrapolated levels, with c* clamped at 0 (the denominator
    K_c + c' read as K_c + c); the nutrient is solved after the phase
    field, so its coefficients use phi^{n+1}.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy import fft as sfft

FLOW_POISEUILLE = 0
FLOW_SHEAR = 1
MOMENTUM_SPLIT = 0      # constant eta_bar implicit, the rest of the stress explicit (Eq. 4.2)
MOMENTUM_IMPLICIT = 1   # the whole variable stress div(2 eta D(v)) by Crank-Nicolson
ENERGY_FLORY_HUGGINS = 0
ENERGY_DOUBLE_WELL = 1


class DomainError(ValueError):
    """The extrapolated phi left (0, 1), where the log energy is undefined."""


class NotConverged(RuntimeError):
    pass


# --------------------------------------------------------------------------
# Grid (§4: structured uniform grid, nodes (i dx, j dy))

@dataclass
class Grid:
    nx: int
    ny: int
    lx: float
    ly: float

    @property
    def hx(self):
        return self.lx / self.nx

    @property
    def hy(self):
        return self.ly / self.ny

    @property
    def shape(self):
        return (self.ny + 1, self.nx)

    @property
    def w(self):
        w = np.ones(self.shape)
        w[0, :] = 0.5
        w[-1, :] = 0.5
        return w


def grid_of(prm) -> Grid:
    return Grid(prm.nx, prm.ny, prm.lx, prm.ly)


def wdot(g: Grid, x, y):
    return float(np.sum(g.w * x * y))


def wnorm(g: Grid, x):
    return math.sqrt(wdot(g, x, x))


def mass(g: Grid, phi):
    """<phi, 1>_W: the discrete mass conserved by Eq. 2.4 with zero flux."""
    return float(np.sum(g.w * phi))


# ghost rows ---------------------------------------------------------------

def even_rows(x, depth=1):
    """x with `depth` ghost rows above and below, even reflection about the
    wall rows: x_{-k} = x_k, x_{ny+k} = x_{ny-k} (Eq. 4.7)."""
    top = x[depth:0:-1]
    bot = x[-2:-2 - depth:-1]
    return np.concatenate([top, x, bot], axis=0)


def odd_rows(x):
    """x with one ghost row each side, odd reflection x_{-1} = -x_1 (used for
    the wall-normal flux, which vanishes on the walls)."""
    return np.concatenate([-x[1:2], x, -x[-2:-1]], axis=0)


def xp(x):  # x_{i+1} (periodic, §4.1 index wrap)
    return np.roll(x, -1, axis=1)


def xm(x):  # x_{i-1}
    return np.roll(x, 1, axis=1)


# --------------------------------------------------------------------------
# Spatial operators (§4, central differences)

def lap(g: Grid, x):
    """L_h x = -Laplacian_h x: the 5-point row (4, -1, -1, -1, -1) of
    Listing 3 scaled by the mesh widths, x periodic, walls by even ghost
    rows (zero normal derivative, Eq. 4.6/4.7)."""
    e = even_rows(x)
    s, c, n = e[:-2], e[1:-1], e[2:]
    return (2.0 * c - xm(c) - xp(c)) / g.hx ** 2 + (2.0 * c - s - n) / g.hy ** 2


def ga(g: Grid, a, x):
    """G_a x = -div_h(a grad_h x), the conservative 5-point form of the
    mobility term of Eq. 2.4; face values are means of the two nodes, a and
    x reflected evenly at the walls (zero flux, Eq. 4.6)."""
    ae, xe = even_rows(a), even_rows(x)
    a_e = 0.5 * (a + xp(a))
    a_w = 0.5 * (a + xm(a))
    a_n = 0.5 * (a + ae[2:])
    a_s = 0.5 * (a + ae[:-2])
    fx = a_e * (xp(x) - x) - a_w * (x - xm(x))
    fy = a_n * (xe[2:] - x) - a_s * (x - xe[:-2])
    return -(fx / g.hx ** 2 + fy / g.hy ** 2)


def dx_c(g: Grid, f):
    """Central x-derivative (periodic)."""
    return (xp(f) - xm(f)) / (2.0 * g.hx)


def dy_c(g: Grid, f):
    """Central y-derivative on interior rows; zero on the wall rows (the
    value even reflection gives)."""
    out = np.zeros_like(f)
    out[1:-1] = (f[2:] - f[:-2]) / (2.0 * g.hy)
    return out


def div_c(g: Grid, fx, fy):
    """Nodal central divergence D_c(F); the wall-normal component is
    odd-reflected (it vanishes on the walls)."""
    ye = odd_rows(fy)
    return dx_c(g, fx) + (ye[2:] - ye[:-2]) / (2.0 * g.hy)


def grad_c(g: Grid, p):
    """Central gradient of p (Eq. 4.5), wall rows evenly reflected."""
    return dx_c(g, p), dy_c(g, p)


def dxx_face(g: Grid, c, f):
    """d/dx (c df/dx), compact face form with face means of c (periodic)."""
    c_e = 0.5 * (c + xp(c))
    c_w = 0.5 * (c + xm(c))
    return (c_e * (xp(f) - f) - c_w * (f - xm(f))) / g.hx ** 2


def dyy_face(g: Grid, c, f):
    """d/dy (c df/dy), compact face form, interior rows only (0 on walls)."""
    out = np.zeros_like(f)
    cn = 0.5 * (c[1:-1] + c[2:])
    cs = 0.5 * (c[1:-1] + c[:-2])
    out[1:-1] = (cn * (f[2:] - f[1:-1]) - cs * (f[1:-1] - f[:-2])) / g.hy ** 2
    return out


# --------------------------------------------------------------------------
# Free energy (Eq. 2.3 / 3.3 and the Flory-Huggins reading)

def f_bulk(prm, phi):
    if prm.energy == ENERGY_DOUBLE_WELL:
        return prm.gamma2 * phi ** 2 * (1.0 - phi) ** 2
    return (phi * np.log(phi) / prm.n_poly + (1.0 - phi) * np.log(1.0 - phi)
            + prm.chi * phi * (1.0 - phi))


def f_prime(prm, phi):
    """F'(phi): the bulk part of the chemical potential delta f / delta phi."""
    if prm.energy == ENERGY_DOUBLE_WELL:
        return 2.0 * prm.gamma2 * phi * (1.0 - phi) * (1.0 - 2.0 * phi)
    return ((np.log(phi) + 1.0) / prm.n_poly - np.log(1.0 - phi) - 1.0
            + prm.chi * (1.0 - 2.0 * phi))


def energy(prm, g: Grid, phi):
    """E_h = hx hy [ (kappa/2) <phi, L_h phi>_W + <F(phi), 1>_W ], with the
    gradient part written as the sum of squared forward differences."""
    dxf = (xp(phi) - phi) / g.hx
    dyf = (phi[1:] - phi[:-1]) / g.hy
    grad2 = np.sum(g.w * dxf ** 2) + np.sum(dyf ** 2)
    return g.hx * g.hy * (0.5 * prm.kappa * grad2 + np.sum(g.w * f_bulk(prm, phi)))


# --------------------------------------------------------------------------
# The three linear operators solved each step

def ch_apply(prm, g: Grid, a, x):
    """A_phi x = x/dt + 1/2 G_a (kappa L_h x + S x): the Crank-Nicolson
    matrix of Eq. 2.4 (fourth order, 13-point; wide stencil of §1)."""
    psi = prm.kappa * lap(g, x) + prm.stab_s * x
    return x / prm.dt + 0.5 * ga(g, a, psi)


def eta_bar(prm):
    return max(prm.eta_water, prm.eta_biofilm)


def rho0(prm):
    if prm.rho_water != prm.rho_biofilm:
        raise ValueError("variable density is not supported")
    return prm.rho_water


def helm_apply(prm, g: Grid, x):
    """H x for the velocity predictor (Eq. 4.3): rho/dt x + eta_bar/2 L_h x
    on interior rows (wall neighbours as stored), rho/dt x on wall rows
    (Dirichlet rows, decoupled)."""
    c0 = rho0(prm) / prm.dt
    nu = 0.5 * eta_bar(prm)
    y = c0 * x
    c = x[1:-1]
    y[1:-1] += nu * ((2.0 * c - xm(c) - xp(c)) / g.hx ** 2
                     + (2.0 * c - x[:-2] - x[2:]) / g.hy ** 2)
    return y


def poisson_apply(prm, g: Grid, x):
    """L_h p (Eq. 4.4 with constant density): singular, zero-flux walls."""
    return lap(g, x)


def nut_coefficients(prm, phi_new, phi_old):
    """Coefficients of the nutrient system (Eq. 2.6-2.7, CN): the diagonal
    phi_s^{n+1}/dt + A/2 phi^{n+1/2} and the nodal diffusion coefficient
    D_s phi_s^{n+1/2}; also phi^{n+1/2}."""
    ph = 0.5 * (phi_new + phi_old)
    diag = (1.0 - phi_new) / prm.dt + 0.5 * prm.consume_a * ph
    ks = prm.diff_s * (1.0 - ph)
    return diag, ks, ph


def nut_domain_check(prm, phi_new, phi_old):
    """The nutrient lives in the solvent fraction phi_s = 1 - phi (Eq. 2.6):
    K is positive definite only while phi_s^{n+1} > 0 and the diffusion
    coefficient D_s phi_s^{n+1/2} >= 0, so a step whose corrected phi^{n+1}
    reaches 1 stops before the nutrient solve."""
    _, ks, _ = nut_coefficients(prm, phi_new, phi_old)
    if np.any(~(1.0 - phi_new > 0.0)) or np.any(~(ks >= 0.0)):
        raise DomainError("phi^{n+1} >= 1: the solvent fraction of the nutrient vanishes")


def nut_apply(prm, g: Grid, phi_new, phi_old, x):
    """K x = diag x + 1/2 G_k x, k = D_s phi_s^{n+1/2}, zero flux on both
    walls (G_k reflects evenly).  With c = c_bulk on the top wall the top
    row is the Dirichlet row x/dt instead (row ny-1 keeps the stored top
    row as its neighbour)."""
    diag, ks, _ = nut_coefficients(prm, phi_new, phi_old)
    y = diag * x + 0.5 * ga(g, ks, x)
    if nut_dirichlet_top(prm):
        y[-1] = x[-1] * (1.0 / prm.dt)
    return y


def nut_rhs(prm, g: Grid, st: State, phi_new):
    """Right-hand side of the nutrient system: (phi_s^n/dt - A/2 phi^{n+1/2})
    c^n - 1/2 G_k c^n - D_c(c* phi_s* v*) (the wall-normal flux odd about
    both walls); c_bulk/dt on the top wall when it is a Dirichlet row."""
    _, ks, ph = nut_coefficients(prm, phi_new, st.phi)
    cs = extrapolate(st.c, st.c_prev)
    pss = 1.0 - extrapolate(st.phi, st.phi_prev)
    us = extrapolate(st.u, st.u_prev)
    vs = extrapolate(st.v, st.v_prev)
    b = (((1.0 - st.phi) / prm.dt - 0.5 * prm.consume_a * ph) * st.c
         - 0.5 * ga(g, ks, st.c) - div_c(g, cs * pss * us, cs * pss * vs))
    if nut_dirichlet_top(prm):
        b[-1] = prm.c_bulk * (1.0 / prm.dt)
    return b


# --------------------------------------------------------------------------
# Krylov solvers (§4.1, Listing 4: GMRES with a Jacobi preconditioner)

def probe_diagonal(apply, shape, radius=2):
    """Diagonal of a stencil operator of the given radius by probing with
    coloured indicator vectors (colours repeat every 2r+1 rows and every
    period of columns that divides nx, so no two nodes of one colour share a
    stencil)."""
    ny1, nx = shape
    cy = 2 * radius + 1
    cx = nx
    for c in range(2 * radius + 1, nx + 1):
        if nx % c == 0:
            cx = c
            break
    d = np.zeros(shape)
    J, I = np.indices(shape)
    for ky in range(cy):
        for kx in range(cx):
            e = ((J % cy == ky) & (I % cx == kx)).astype(np.float64)
            d += e * apply(e)
    return d


def gmres(g: Grid, apply, b, x0=None, restart=30, rtol=1e-14, maxit=5000,
          diag=None):
    """Restarted GMRES(m), right-preconditioned by Jacobi (Listing 4), in
    the W inner product; modified Gram-Schmidt and Givens rotations.
    Stops when ||b - A x||_W <= rtol ||b||_W (checked on the true
    residual at every restart)."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    dinv = np.ones_like(b) if diag is None else 1.0 / diag
    bn = wnorm(g, b)
    if bn == 0.0:
        return np.zeros_like(b), 0
    its = 0
    last = math.inf
    while True:
        r = b - apply(x)
        beta = wnorm(g, r)
        if beta <= rtol * bn:
            return x, its
        if its >= maxit or beta >= 0.999 * last:
            raise NotConverged(f"gmres: {beta / bn:.3e} after {its}")
        last = beta
        V = [r / beta]
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        s = np.zeros(restart + 1)
        s[0] = beta
        k_used = 0
        for k in range(restart):
            w = apply(dinv * V[k])
            for i in range(k + 1):
                H[i, k] = wdot(g, w, V[i])
                w = w - H[i, k] * V[i]
            hk1 = wnorm(g, w)
            H[k + 1, k] = hk1
            for i in range(k):
                t = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
                H[i + 1, k] = -sn[i] * H[i, k] + cs[i] * H[i + 1, k]
                H[i, k] = t
            den = math.hypot(H[k, k], H[k + 1, k])
            cs[k], sn[k] = H[k, k] / den, H[k + 1, k] / den
            H[k, k] = den
            H[k + 1, k] = 0.0
            s[k + 1] = -sn[k] * s[k]
            s[k] = cs[k] * s[k]
            its += 1
            k_used = k + 1
            if hk1 == 0.0 or abs(s[k + 1]) <= rtol * bn or its >= maxit:
                break
            V.append(w / hk1)
        y = np.linalg.solve(np.triu(H[:k_used, :k_used]), s[:k_used])
        upd = sum(y[i] * V[i] for i in range(k_used))
        x = x + dinv * upd


def cg(g: Grid, apply, b, x0=None, rtol=1e-14, maxit=100000, diag=None,
       project=False):
    """Preconditioned conjugate gradients in the W inner product (the
    operators are W-symmetric).  `project` keeps iterates W-orthogonal to
    the constants (the singular pressure problem, Listing 5)."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    dinv = np.ones_like(b) if diag is None else 1.0 / diag
    sw = float(np.sum(g.w))

    def proj(z):
        return z - mass(g, z) / sw if project else z

    r = proj(b - apply(x))
    bn = wnorm(g, b)
    if bn == 0.0:
        return np.zeros_like(b), 0
    z = proj(dinv * r)
    p = z.copy()
    rz = wdot(g, r, z)
    for it in range(1, maxit + 1):
        q = apply(p)
        alpha = rz / wdot(g, p, q)
        x = x + alpha * p
        r = r - alpha * q
        if wnorm(g, r) <= rtol * bn:
            return proj(x), it
        z = proj(dinv * r)
        rz_new = wdot(g, r, z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    raise NotConverged("cg")


# --------------------------------------------------------------------------
# Exact solves (a library FFT as a step): constant-coefficient operators are
# diagonal in the cos/sin x Fourier basis, so these give the exact discrete
# solution the paper's iterative solves converge to.

def _lam_x(g: Grid):
    k = np.arange(g.nx)
    return 4.0 / g.hx ** 2 * np.sin(np.pi * k / g.nx) ** 2


def _lam_y_neumann(g: Grid):
    l = np.arange(g.ny + 1)
    return 4.0 / g.hy ** 2 * np.sin(np.pi * l / (2 * g.ny)) ** 2


def _lam_y_dirichlet(g: Grid):
    l = np.arange(1, g.ny)
    return 4.0 / g.hy ** 2 * np.sin(np.pi * l / (2 * g.ny)) ** 2


def neumann_spectral_solve(g: Grid, b, symbol):
    """Solve S(L_x, L_y) x = b for an operator diagonal in the basis
    cos(pi l j / ny) e^{2 pi i k i / nx} (DCT-I in y, FFT in x).  `symbol`
    maps (lam_x, lam_y) grids to eigenvalues; zero eigenvalues are treated
    as the null space (coefficient set to zero)."""
    B = sfft.dct(sfft.fft(b, axis=1), type=1, axis=0)
    lam = symbol(_lam_x(g)[None, :], _lam_y_neumann(g)[:, None])
    with np.errstate(divide="ignore", invalid="ignore"):
        X = np.where(lam == 0.0, 0.0, B / np.where(lam == 0.0, 1.0, lam))
    return np.real(sfft.ifft(sfft.idct(X, type=1, axis=0), axis=1))


def poisson_solve(prm, g: Grid, d):
    """Exact solution of L_h p = d - <d,1>_W/<1,1>_W with <p,1>_W = 0."""
    dproj = d - mass(g, d) / float(np.sum(g.w))
    return neumann_spectral_solve(g, dproj, lambda lx, ly: lx + ly)


def helm_solve(prm, g: Grid, b):
    """Exact solution of H x = b (velocity predictor): the wall rows give
    x = b dt / rho; their values are lifted into the interior right-hand
    side, which is solved by DST-I in y and FFT in x."""
    c0 = rho0(prm) / prm.dt
    nu = 0.5 * eta_bar(prm)
    x = np.empty_like(b)
    x[0] = b[0] / c0
    x[-1] = b[-1] / c0
    rhs = b[1:-1].copy()
    rhs[0] += nu * x[0] / g.hy ** 2
    rhs[-1] += nu * x[-1] / g.hy ** 2
    B = sfft.dst(sfft.fft(rhs, axis=1), type=1, axis=0)
    lam = c0 + nu * (_lam_x(g)[None, :] + _lam_y_dirichlet(g)[:, None])
    x[1:-1] = np.real(sfft.ifft(sfft.idst(B / lam, type=1, axis=0), axis=1))
    return x


def ch_const_solve(prm, g: Grid, a_const, b):
    """Exact solution of A_phi x = b when the mobility coefficient a is a
    constant (then G_a = a L_h and A_phi is diagonal in the Neumann basis)."""
    k, s, dt = prm.kappa, prm.stab_s, prm.dt
    return neumann_spectral_solve(
        g, b, lambda lx, ly: 1.0 / dt + 0.5 * a_const * (lx + ly) * (k * (lx + ly) + s))


# --------------------------------------------------------------------------
# Dense brute force (tiny grids)

def assemble(apply, shape):
    n = shape[0] * shape[1]
    A = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        A[:, k] = apply(e.reshape(shape)).ravel()
    return A


def dense_solve(apply, shape, b):
    return np.linalg.solve(assemble(apply, shape), b.ravel()).reshape(shape)


def dense_poisson_solve(g: Grid, d):
    """Bordered system [L_h  1; w^T 0] [p; lambda] = [d_proj; 0]."""
    shape = g.shape
    n = shape[0] * shape[1]
    A = assemble(lambda x: lap(g, x), shape)
    M = np.zeros((n + 1, n + 1))
    M[:n, :n] = A
    M[:n, n] = 1.0
    M[n, :n] = g.w.ravel()
    dproj = d - mass(g, d) / float(np.sum(g.w))
    rhs = np.concatenate([dproj.ravel(), [0.0]])
    return np.linalg.solve(M, rhs)[:n].reshape(shape)


# --------------------------------------------------------------------------
# One time step (§4: CH first, then the projection method, Eq. 4.3-4.5)

@dataclass
class State:
    phi: np.ndarray
    phi_prev: np.ndarray
    u: np.ndarray
    u_prev: np.ndarray
    v: np.ndarray
    v_prev: np.ndarray
    p: np.ndarray
    m0: float
    step: int = 0
    iters: dict = field(default_factory=dict)
    c: np.ndarray = None        # nutrient c^n and c^{n-1} (None: nutrient off)
    c_prev: np.ndarray = None

    def copy(self):
        cp = lambda a: None if a is None else a.copy()
        return State(self.phi.copy(), self.phi_prev.copy(), self.u.copy(),
                     self.u_prev.copy(), self.v.copy(), self.v_prev.copy(),
                     self.p.copy(), self.m0, self.step, dict(self.iters),
                     cp(self.c), cp(self.c_prev))


def init_state(prm, phi0, u0, v0, p0, c0=None) -> State:
    """Start of a run: previous levels equal to the current ones; the
    nutrient (when on) starts at c0, previous level c0 as well."""
    g = grid_of(prm)
    c = None
    if nutrient_on(prm):
        if c0 is None:
            raise ValueError("the nutrient is on: c0 is required")
        c = c0.copy()
    return State(phi0.copy(), phi0.copy(), u0.copy(), u0.copy(), v0.copy(),
                 v0.copy(), p0.copy(), mass(g, phi0), c=c,
                 c_prev=None if c is None else c.copy())


NUT_BC_ZERO_FLUX = 0   # zero total flux on both walls (the boundary block of §2)
NUT_BC_BULK_TOP = 1    # c = c_bulk on the top wall, zero flux on the substratum


def nutrient_on(prm) -> bool:
    return bool(getattr(prm, "nutrient", 0))


def nut_dirichlet_top(prm) -> bool:
    return getattr(prm, "nutrient_bc", NUT_BC_ZERO_FLUX) == NUT_BC_BULK_TOP


def extrapolate(q, q_prev):
    """q* = (3 q^n - q^{n-1}) / 2 (the n+1/2 extrapolation, §4)."""
    return 1.5 * q - 0.5 * q_prev


def ch_coefficient(prm, st: State):
    """a = M phi*: the degenerate mobility of Eq. 2.4 at the extrapolated
    phase field."""
    phis = extrapolate(st.phi, st.phi_prev)
    if np.any(phis <= 0.0) or np.any(phis >= 1.0):
        raise DomainError("extrapolated phi outside (0, 1)")
    return prm.mobility * phis, phis


def growth(prm, phis, cs):
    """Network production g_n = eps_g mu phi c / (K_c + c) (Eq. 2.5) at the
    extrapolated levels phi*, c*, with c* clamped at 0."""
    c = np.maximum(cs, 0.0)
    return prm.growth_eps * prm.growth_mu * phis * c / (prm.growth_kc + c)


def ch_rhs(prm, g: Grid, st: State):
    """b_phi = phi^n/dt - 1/2 G_a(kappa L_h + S) phi^n - G_a(F'(phi*) - S phi*)
    - D_c(phi* v*) + g_n*  (Eq. 2.4 with CN + extrapolation; g_n = 0 unless
    the nutrient is on).  Returns (b, a, g_n*)."""
    a, phis = ch_coefficient(prm, st)
    us = extrapolate(st.u, st.u_prev)
    vs = extrapolate(st.v, st.v_prev)
    psi_n = prm.kappa * lap(g, st.phi) + prm.stab_s * st.phi
    q = f_prime(prm, phis) - prm.stab_s * phis
    b = (st.phi / prm.dt - 0.5 * ga(g, a, psi_n) - ga(g, a, q)
         - div_c(g, phis * us, phis * vs))
    gn = np.zeros_like(b)
    if nutrient_on(prm):
        gn = growth(prm, phis, extrapolate(st.c, st.c_prev))
        b = b + gn
    return b, a, gn


def body_force_x(prm):
    if prm.flow_mode == FLOW_POISEUILLE:
        return 8.0 * prm.eta_water * prm.u_max / prm.ly ** 2
    return 0.0


def wall_u(prm):
    """(u on y = 0, u on y = Ly) for the predictor's Dirichlet rows."""
    if prm.flow_mode == FLOW_POISEUILLE:
        return 0.0, 0.0
    return 0.0, prm.u_max


def capillary_force(prm, g: Grid, ph):
    """-Gamma div(grad phi (x) grad phi) at phi^{n+1/2} (Eq. 4.1, the
    divergence lost in Eq. 3.3 restored), central differences; the
    wall-normal derivative of phi is zero on the walls (Eq. 4.6)."""
    gam = prm.gamma_cap
    gx, gy = dx_c(g, ph), dy_c(g, ph)
    cx = -gam * (dx_c(g, gx * gx) + dy_c(g, gx * gy))
    cy = -gam * (dx_c(g, gx * gy) + dy_c(g, gy * gy))
    return cx, cy


def viscous_remainder(g: Grid, ep, us, vs):
    """The explicit part of the variable viscous stress, div(2 eta' D(v*))
    with eta' = eta - eta_bar (Eq. 4.1-4.2), in the form it takes for a
    divergence-free field: div(eta' grad v*) + (grad v*)^T grad eta'."""
    ex, ey = dx_c(g, ep), dy_c(g, ep)
    vx = (dxx_face(g, ep, us) + dyy_face(g, ep, us)
          + ex * dx_c(g, us) + ey * dx_c(g, vs))
    vy = (dxx_face(g, ep, vs) + dyy_face(g, ep, vs)
          + ex * dy_c(g, us) + ey * dy_c(g, vs))
    return vx, vy


def convection(g: Grid, us, vs):
    """(v* . grad) v*, central differences (Eq. 4.2)."""
    conv_u = us * dx_c(g, us) + vs * dy_c(g, us)
    conv_v = us * dx_c(g, vs) + vs * dy_c(g, vs)
    return conv_u, conv_v


def momentum_rhs(prm, g: Grid, st: State, phi_new):
    """Right-hand sides of the two predictor systems (Eq. 4.1-4.3):
    rho u^n/dt - rho (v*.grad) u* - eta_bar/2 L_h u^n + R + f on interior
    rows, with R = -Gamma div(grad phi grad phi) + div(2 (eta - eta_bar)
    D(v*)) at phi^{n+1/2} (viscous part in its divergence-free form); rho/dt
    times the wall value on wall rows."""
    rho = rho0(prm)
    ph = 0.5 * (phi_new + st.phi)
    us = extrapolate(st.u, st.u_prev)
    vs = extrapolate(st.v, st.v_prev)
    eta = ph * prm.eta_biofilm + (1.0 - ph) * prm.eta_water
    ep = eta - eta_bar(prm)
    nu = 0.5 * eta_bar(prm)
    cx, cy = capillary_force(prm, g, ph)
    vx, vy = viscous_remainder(g, ep, us, vs)
    conv_u, conv_v = convection(g, us, vs)

    def lap_int(f):
        out = np.zeros_like(f)
        c = f[1:-1]
        out[1:-1] = ((2.0 * c - xm(c) - xp(c)) / g.hx ** 2
                     + (2.0 * c - f[:-2] - f[2:]) / g.hy ** 2)
        return out

    bu = rho * st.u / prm.dt - rho * conv_u - nu * lap_int(st.u) + cx + vx + body_force_x(prm)
    bv = rho * st.v / prm.dt - rho * conv_v - nu * lap_int(st.v) + cy + vy
    ub0, ubn = wall_u(prm)
    c0 = rho / prm.dt
    bu[0], bu[-1] = c0 * ub0, c0 * ubn
    bv[0], bv[-1] = 0.0, 0.0
    return bu, bv


# --------------------------------------------------------------------------
# Fully implicit variable-viscosity momentum (the stress of Eq. 4.1 without
# the eta_bar split): Crank-Nicolson on div(2 eta D(v)), eta at phi^{n+1/2},
# u and v coupled through the cross derivatives.

def momentum_implicit(prm) -> bool:
    return getattr(prm, "momentum", MOMENTUM_SPLIT) == MOMENTUM_IMPLICIT


def viscous_stress_div(g: Grid, eta, u, v):
    """div(2 eta D(v)), D = (grad v + grad v^T)/2, on interior rows (0 on the
    walls): d/dx(2 eta u_x) + d/dy(eta u_y) + d/dy(eta v_x) and
    d/dx(eta u_y) + d/dx(eta v_x) + d/dy(2 eta v_y).  The normal-normal and
    tangential second derivatives take the compact face-mean form, the cross
    derivatives central differences of central differences; wall rows hold
    the stored wall values."""
    tu = dxx_face(g, 2.0 * eta, u) + dyy_face(g, eta, u) + dy_c(g, eta * dx_c(g, v))
    tv = dx_c(g, eta * dy_c(g, u)) + dxx_face(g, eta, v) + dyy_face(g, 2.0 * eta, v)
    for t in (tu, tv):
        t[0] = 0.0
        t[-1] = 0.0
    return tu, tv


def viscosity(prm, ph):
    """eta(phi) = phi eta_biofilm + (1 - phi) eta_water."""
    return ph * prm.eta_biofilm + (1.0 - ph) * prm.eta_water


def visc_apply(prm, g: Grid, eta, u, v):
    """The implicit momentum matrix: rho/dt v - 1/2 div(2 eta D(v)) on interior
    rows, rho/dt v on the wall rows (Dirichlet rows, decoupled)."""
    c0 = rho0(prm) / prm.dt
    tu, tv = viscous_stress_div(g, eta, u, v)
    return c0 * u - 0.5 * tu, c0 * v - 0.5 * tv


def momentum_rhs_implicit(prm, g: Grid, st: State, phi_new):
    """Right-hand sides of the coupled system: rho u^n/dt - rho (v*.grad) u*
    + 1/2 div(2 eta D(v^n)) - Gamma div(grad phi grad phi) + f on interior
    rows, eta and the capillary force at phi^{n+1/2}; rho/dt times the wall
    value on wall rows."""
    rho = rho0(prm)
    ph = 0.5 * (phi_new + st.phi)
    us = extrapolate(st.u, st.u_prev)
    vs = extrapolate(st.v, st.v_prev)
    eta = viscosity(prm, ph)
    cx, cy = capillary_force(prm, g, ph)
    conv_u, conv_v = convection(g, us, vs)
    tu, tv = viscous_stress_div(g, eta, st.u, st.v)
    bu = rho * st.u / prm.dt - rho * conv_u + 0.5 * tu + cx + body_force_x(prm)
    bv = rho * st.v / prm.dt - rho * conv_v + 0.5 * tv + cy
    ub0, ubn = wall_u(prm)
    c0 = rho / prm.dt
    bu[0], bu[-1] = c0 * ub0, c0 * ubn
    bv[0], bv[-1] = 0.0, 0.0
    return bu, bv, eta


def visc_diagonal(prm, g: Grid, eta):
    """Diagonals of the two blocks of visc_apply (the cross terms have none)."""
    c0 = rho0(prm) / prm.dt
    fe, fw = 0.5 * (eta + xp(eta)), 0.5 * (eta + xm(eta))
    fn, fs = np.ones_like(eta), np.ones_like(eta)
    fn[1:-1] = 0.5 * (eta[1:-1] + eta[2:])
    fs[1:-1] = 0.5 * (eta[1:-1] + eta[:-2])
    du = c0 + 0.5 * (2.0 * (fe + fw) / g.hx ** 2 + (fn + fs) / g.hy ** 2)
    dv = c0 + 0.5 * ((fe + fw) / g.hx ** 2 + 2.0 * (fn + fs) / g.hy ** 2)
    du[0] = du[-1] = dv[0] = dv[-1] = c0
    return du, dv


def visc_solve(prm, g: Grid, eta, bu, bv, method="cg", rtol=1e-14):
    """Solve the coupled system: the wall rows directly (u = b/c0), the
    interior by dense LU (tiny grids) or Jacobi-preconditioned CG on the
    stacked unknowns (the matrix is symmetric positive definite on the
    fields that vanish on the walls)."""
    c0 = rho0(prm) / prm.dt
    ny1 = g.ny + 1
    stack = lambda a, b: np.concatenate([a, b], axis=0)

    def apply(x):
        yu, yv = visc_apply(prm, g, eta, x[:ny1], x[ny1:])
        return stack(yu, yv)

    b = stack(bu, bv)
    if method == "lu":
        x = dense_solve(apply, b.shape, b)
        return x[:ny1], x[ny1:]
    x0 = np.zeros_like(b)
    for r in (0, g.ny, ny1, ny1 + g.ny):
        x0[r] = b[r] / c0
    du, dv = visc_diagonal(prm, g, eta)
    sg = Grid(g.nx, 2 * g.ny + 1, g.lx, g.ly)   # weights: wall rows of the residual vanish
    x, _ = cg(sg, apply, b, x0=x0, rtol=rtol, diag=stack(du, dv))
    return x[:ny1], x[ny1:]


def solve_phi(prm, g, a, b, x0=None, method="gmres", rtol=1e-14):
    apply = lambda x: ch_apply(prm, g, a, x)
    if method == "lu":
        return dense_solve(apply, g.shape, b), 0
    diag = probe_diagonal(apply, g.shape)
    return gmres(g, apply, b, x0=x0, restart=30, rtol=rtol, diag=diag)


def solve_nut(prm, g, phi_new, phi_old, b, x0=None, method="cg", rtol=1e-14):
    """Solve K c = b: dense LU (tiny grids) or Jacobi-preconditioned CG in
    the W inner product.  K is W-symmetric positive definite (with a
    Dirichlet top row: on the fields whose top row is zero; the initial
    guess then carries that row, so every residual and search direction
    stays in that space)."""
    apply = lambda x: nut_apply(prm, g, phi_new, phi_old, x)
    if method == "lu":
        return dense_solve(apply, g.shape, b), 0
    x = np.zeros_like(b) if x0 is None else x0.copy()
    if nut_dirichlet_top(prm):
        x[-1] = b[-1] * prm.dt
    diag = probe_diagonal(apply, g.shape, radius=1)
    return cg(g, apply, b, x0=x, rtol=rtol, diag=diag)


def step(prm, st: State, ch_method="gmres", rtol=1e-14) -> State:
    """Advance (phi, u, v, p) by one time step: CH solve, mass correction,
    velocity predictor (Eq. 4.3), pressure Poisson (Eq. 4.4), velocity
    correction (Eq. 4.5); with the nutrient on, also c (Eq. 2.6)."""
    g = grid_of(prm)
    rho = rho0(prm)
    # 1-2. Cahn-Hilliard system
    b, a, gn = ch_rhs(prm, g, st)
    phi_new, its = solve_phi(prm, g, a, b, x0=st.phi, method=ch_method, rtol=rtol)
    # 3. mass correction (the target grows by dt <g_n, 1>_W)
    target = st.m0 + prm.dt * mass(g, gn) if nutrient_on(prm) else st.m0
    phi_new = phi_new + (target - mass(g, phi_new)) / float(np.sum(g.w))
    c_new = None
    if nutrient_on(prm):
        nut_domain_check(prm, phi_new, st.phi)
        bc = nut_rhs(prm, g, st, phi_new)
        c_new, _ = solve_nut(prm, g, phi_new, st.phi, bc, x0=st.c, rtol=rtol)
    # 4-5. velocity predictor
    if momentum_implicit(prm):
        bu, bv, eta = momentum_rhs_implicit(prm, g, st, phi_new)
        u_pred, v_pred = visc_solve(prm, g, eta, bu, bv, rtol=rtol)
    else:
        bu, bv = momentum_rhs(prm, g, st, phi_new)
        u_pred = helm_solve(prm, g, bu)
        v_pred = helm_solve(prm, g, bv)
    # 6. pressure
    d = rho * div_c(g, u_pred, v_pred)
    p = poisson_solve(prm, g, d)
    # 7. correction on interior rows
    px, py = grad_c(g, p)
    u_new = u_pred.copy()
    v_new = v_pred.copy()
    u_new[1:-1] += px[1:-1] / rho
    v_new[1:-1] += py[1:-1] / rho
    out = State(phi_new, st.phi, u_new, st.u, v_new, st.v, p, target, st.step + 1,
                {"phi": its}, c_new, st.c)
    return out


def run(prm, phi0, u0, v0, p0, nsteps, c0=None, **kw) -> State:
    st = init_state(prm, phi0, u0, v0, p0, c0)
    for _ in range(nsteps):
        st = step(prm, st, **kw)
    return st


# --------------------------------------------------------------------------
# Single solves with frozen coefficients (counterparts of cahn_solve)

def solve_system(prm, st: State, system: str, rhs):
    """Exact solution of one of the systems at the state's coefficients:
    'phi' (A_phi with a = M phi*), 'u'/'v' (H), 'p' (L_h, projected rhs,
    <p,1>_W = 0), 'c' (the nutrient K with phi^{n+1} = phi^n = phi)."""
    g = grid_of(prm)
    if system == "c":
        x, _ = solve_nut(prm, g, st.phi, st.phi, rhs, rtol=1e-14)
        return x
    if system == "phi":
        a, _ = ch_coefficient(prm, st)
        x, _ = solve_phi(prm, g, a, rhs, rtol=1e-14)
        return x
    if system in ("u", "v"):
        return helm_solve(prm, g, rhs)
    if system == "p":
        return poisson_solve(prm, g, rhs)
    raise ValueError(system)
