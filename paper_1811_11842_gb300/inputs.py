"""Seeded synthetic inputs shared by the CUDA path, its tests and the oracle.

This module holds no arithmetic of the solver: only the problem record
(grid, parameters, solver options), a counter-based random generator and the
initial-condition recipe.  The same arrays are handed, bit for bit, to the
CUDA library and to the CPU oracle.

Problem statement (grid, parameters, phi, velocity, pressure, dt) follows the
paper's §3 (dimensionless parameters, Eq. 3.2) and §4 (uniform nodal grid
x_i = i*dx, y_j = j*dy; periodic in x, walls at y = 0 and y = Ly).

Initial condition (the paper gives its "mushroom shaped protrusions" only as a
figure, §5.1 / Fig. 5): a base layer of height h_b plus semicircular
protrusions, smoothed by a tanh profile of width eps, plus uniform noise.
phi_in / phi_out are the two binodal compositions of the Flory-Huggins
energy (symmetric case N = 1); the random numbers come from SplitMix64
(Steele, Lea & Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014) in row-major node order.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence

import numpy as np

# flow modes, precisions, Krylov choices, energies (values mirror include/cahn.h)
FLOW_POISEUILLE = 0
FLOW_SHEAR = 1
FP64 = 0
MIXED = 1
GMRES = 0
BICGSTAB = 1
ENERGY_FLORY_HUGGINS = 0
ENERGY_DOUBLE_WELL = 1
MOMENTUM_SPLIT = 0
MOMENTUM_IMPLICIT = 1
PC_MG = 0
PC_JACOBI = 1
PC_SCHWARZ = 2


@dataclasses.dataclass
class Params:
    """One instance's grid, physical parameters and solver options."""
    nx: int = 64            # periodic columns (intervals in x)
    ny: int = 64            # intervals in y; ny + 1 rows including both walls
    lx: float = 2.0
    ly: float = 1.0
    eps: float = 0.02       # interface width; kappa = eps**2
    mobility: float = 1e-3  # M in the degenerate mobility a = M * phi
    chi: float = 2.5        # Flory-Huggins interaction parameter
    n_poly: float = 1.0     # generalised polymerisation N
    stab_s: float = 0.0     # stabilisation S >= 0 (0 = plain extrapolation)
    eta_water: float = 1.0
    eta_biofilm: float = 10.0
    rho_water: float = 1.0
    rho_biofilm: float = 1.0
    gamma_cap: float = 4e-4  # capillary coefficient (defaults to kappa)
    flow_mode: int = FLOW_POISEUILLE
    u_max: float = 1.0
    dt: float = 1e-4
    precision: int = FP64
    krylov: int = GMRES
    restart: int = 30
    mg_levels: int = 5
    max_iters: int = 20000
    rtol: float = 1e-12
    energy: int = ENERGY_FLORY_HUGGINS
    gamma2: float = 0.0     # double-well strength (ENERGY_DOUBLE_WELL only)
    precond: int = 0        # 0 multigrid V-cycle, 1 Jacobi, 2 one-level domain decomposition
    use_graph: int = 0      # 1: CUDA-graph replay with device-side loops
    # nutrient transport and network production (Eq. 2.5-2.7); the defaults
    # are the paper's dimensionless values (§5: D_s, mu, K_c, A)
    nutrient: int = 0       # 1: transport c and add g_n to the phase field
    diff_s: float = 2.3     # D_s
    growth_mu: float = 0.14  # mu, maximum production rate
    growth_kc: float = 0.15  # K_c, half-saturation constant
    growth_eps: float = 1.0  # epsilon, scaling constant of g_n
    consume_a: float = 100.0  # A, consumption g_c = A phi c
    c_bulk: float = 1.0     # initial c; c on the top wall when nutrient_bc = 1
    nutrient_bc: int = 0    # 0 zero flux on both walls (§2), 1 c = c_bulk on the top wall
    momentum: int = 0       # 0 the eta_bar split (Eq. 4.2), 1 fully implicit variable viscosity
    ic_width: float = 0.0   # width of the initial tanh profile (0: eps); not a solver input

    @property
    def kappa(self) -> float:
        return self.eps * self.eps

    def replace(self, **kw) -> "Params":
        return dataclasses.replace(self, **kw)


@dataclasses.dataclass
class Protrusions:
    """Base layer height, protrusion centres (x) and radius."""
    h_b: float = 0.1
    centres: Sequence[float] = (1.0,)
    radius: float = 0.1
    noise: float = 1e-3
    seed: int = 0


# --------------------------------------------------------------------------
# SplitMix64 (counter form): output k of seed s is mix(s + (k+1) * GOLDEN).
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """`count` consecutive SplitMix64 outputs (uint64) from position `start`."""
    k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, start: int = 0) -> np.ndarray:
    """53-bit uniform doubles in [0, 1) from SplitMix64."""
    z = splitmix64(seed, count, start)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


# --------------------------------------------------------------------------
def binodal_pair(chi: float, n_poly: float = 1.0):
    """(phi_in, phi_out) used for the biofilm / water phases of the IC.

    For N = 1 the Flory-Huggins binodal is symmetric about 1/2 and phi_in is
    the root above 1/2 of ln(phi / (1 - phi)) = chi (2 phi - 1); found by
    bisection.  Clamped to [0.05, 0.95]; for chi <= 2.05 (binodal collapsing
    towards 1/2) and for N != 1 the pair falls back to (0.9, 0.1)."""
    if n_poly != 1.0 or chi <= 2.05:
        return 0.9, 0.1
    g = lambda p: math.log(p / (1.0 - p)) - chi * (2.0 * p - 1.0)
    lo, hi = 0.5 + 1e-6, 1.0 - 1e-15
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if g(mid) < 0.0:
            lo = mid
        else:
            hi = mid
    p_in = min(max(0.5 * (lo + hi), 0.05), 0.95)
    return p_in, 1.0 - p_in


def grid_coords(prm: Params):
    x = np.arange(prm.nx, dtype=np.float64) * (prm.lx / prm.nx)
    y = np.arange(prm.ny + 1, dtype=np.float64) * (prm.ly / prm.ny)
    return x, y


def protrusion_phi(prm: Params, geo: Protrusions) -> np.ndarray:
    """phi0[j, i] (rows j = 0..ny, columns i = 0..nx-1), float64 row-major."""
    x, y = grid_coords(prm)
    X, Y = np.meshgrid(x, y)
    d = Y - geo.h_b
    for xc in geo.centres:
        dx = X - xc
        dx = dx - prm.lx * np.round(dx / prm.lx)
        d = np.minimum(d, np.sqrt(dx * dx + (Y - geo.h_b) ** 2) - geo.radius)
    p_in, p_out = binodal_pair(prm.chi, prm.n_poly)
    width = prm.ic_width if prm.ic_width > 0.0 else prm.eps
    phi = p_out + (p_in - p_out) * 0.5 * (1.0 - np.tanh(d / width))
    if geo.noise:
        u = uniform01(geo.seed, phi.size).reshape(phi.shape)
        phi = phi + geo.noise * (2.0 * u - 1.0)
    return np.ascontiguousarray(phi)


def initial_velocity(prm: Params):
    """(u0, v0, p0): parabolic channel profile of peak u_max (POISEUILLE) or
    the linear Couette profile with u = u_max on the top wall (SHEAR)."""
    _, y = grid_coords(prm)
    if prm.flow_mode == FLOW_POISEUILLE:
        prof = 4.0 * prm.u_max * y * (prm.ly - y) / (prm.ly * prm.ly)
        prof[0] = 0.0
        prof[-1] = 0.0
    else:
        prof = prm.u_max * y / prm.ly
    u = np.repeat(prof[:, None], prm.nx, axis=1)
    v = np.zeros_like(u)
    p = np.zeros_like(u)
    return np.ascontiguousarray(u), v, p


def initial_state(prm: Params, geo: Protrusions):
    phi = protrusion_phi(prm, geo)
    u, v, p = initial_velocity(prm)
    return phi, u, v, p


def initial_nutrient(prm: Params) -> np.ndarray:
    """c0: the bulk value everywhere (the channel starts saturated)."""
    return np.full((prm.ny + 1, prm.nx), prm.c_bulk, dtype=np.float64)


def random_field(prm: Params, seed: int, lo: float = -1.0, hi: float = 1.0,
                 start: int = 0) -> np.ndarray:
    """A seeded uniform field of the grid's shape (for operator tests)."""
    n = (prm.ny + 1) * prm.nx
    return lo + (hi - lo) * uniform01(seed, n, start).reshape(prm.ny + 1, prm.nx)


# --------------------------------------------------------------------------
# Workload presets (synthetic stand-ins shaped like the paper's runs).

def config_small() -> tuple:
    """64 x 64 intervals over [0,2]x[0,1], chi 2.5, N 1, eps 0.02, M 1e-3,
    viscosity ratio 10:1, dt 1e-4, 20 steps, one protrusion r 0.1 at x 1."""
    prm = Params(nx=64, ny=64, lx=2.0, ly=1.0, eps=0.02, mobility=1e-3,
                 chi=2.5, n_poly=1.0, eta_water=1.0, eta_biofilm=10.0,
                 gamma_cap=0.02 ** 2, u_max=1.0, dt=1e-4, rtol=1e-12,
                 restart=30, mg_levels=4)
    geo = Protrusions(h_b=0.1, centres=(1.0,), radius=0.1, noise=1e-3, seed=0)
    return prm, geo, 20


def config_medium() -> tuple:
    """The small workload at 256 x 256 intervals, dt 2.5e-5, 200 steps."""
    prm, geo, _ = config_small()
    return prm.replace(nx=256, ny=256, dt=2.5e-5, mg_levels=5), geo, 200


def config_large() -> tuple:
    """1024 x 1024 intervals over [0,4]x[0,1], two protrusions r 0.08 at
    x = 1.3 and 2.7, dt 1e-4, 100 steps, GMRES(30) + 5-level multigrid."""
    prm, geo, _ = config_small()
    prm = prm.replace(nx=1024, ny=1024, lx=4.0, ly=1.0, dt=1e-4, restart=30,
                      mg_levels=5)
    geo = Protrusions(h_b=0.1, centres=(1.3, 2.7), radius=0.08, noise=1e-3,
                      seed=0)
    return prm, geo, 100


# The paper's dimensionless parameter set (§5): Reynolds numbers of the
# solvent and the network, mobility, distortional and separation energies.
PAPER_RE_S, PAPER_RE_N = 9.98e-4, 2.33e-9
PAPER_LAMBDA, PAPER_GAMMA1, PAPER_GAMMA2 = 1e-10, 33.467, 1.25e6


def config_paper(n: int = 256) -> tuple:
    """The paper's own parameter set (§5) on its grid (Table 1: M = 256
    intervals) over [0,1]x[0,1]: the double-well energy Gamma2 phi^2 (1-phi)^2
    with Gamma2 = 1.25e6, kappa = Gamma1 = 33.467 (also the capillary
    coefficient), mobility Lambda = 1e-10, viscosities 1/Re_s (water) and
    1/Re_n (biofilm, a ratio of 4.3e5), rho = 1, the shear flow u = 0.1 on
    the top wall (§5.1), two protrusions r 0.08 at x 0.3 and 0.7 on a base
    layer of height 0.1.  dt 0.02 with the stabilisation S = 2 Gamma2 (the
    largest F'' on [0, 1]; at 256^2 the oracle's phi leaves (0, 1) by step 7
    with dt 0.1 and by step 15 with dt 0.05, and stays inside for 60 steps
    with dt 0.02); the initial tanh profile has width 2h (the equilibrium
    interface width sqrt(Gamma1/Gamma2) = 5.2e-3 is 1.3 cells at 256
    intervals).  20 steps."""
    prm = Params(nx=n, ny=n, lx=1.0, ly=1.0, eps=math.sqrt(PAPER_GAMMA1),
                 mobility=PAPER_LAMBDA, chi=2.5, n_poly=1.0, energy=ENERGY_DOUBLE_WELL,
                 gamma2=PAPER_GAMMA2, gamma_cap=PAPER_GAMMA1, stab_s=2.0 * PAPER_GAMMA2,
                 eta_water=1.0 / PAPER_RE_S, eta_biofilm=1.0 / PAPER_RE_N, rho_water=1.0,
                 rho_biofilm=1.0, flow_mode=FLOW_SHEAR, u_max=0.1, dt=0.02, rtol=1e-12,
                 restart=30, mg_levels=5, ic_width=2.0 / n)
    geo = Protrusions(h_b=0.1, centres=(0.3, 0.7), radius=0.08, noise=1e-3, seed=0)
    return prm, geo, 20


def config_nutrient() -> tuple:
    """The small workload with nutrient transport and network production
    on, at the paper's D_s, mu, K_c and A."""
    prm, geo, n = config_small()
    return prm.replace(nutrient=1), geo, n


BATCH_SIZES = (128, 192, 256, 384, 512)


def config_batch(count: int = 64, seed: int = 0) -> List[tuple]:
    """`count` independent instances; per instance, in order, the generator
    draws the grid size from BATCH_SIZES, chi ~ U[2, 3], log10 M ~ U[-4, -2]
    and the protrusion radius ~ U[0.05, 0.15].  Domain [0,2]x[0,1]."""
    base, geo0, _ = config_small()
    draws = uniform01(seed, 4 * count, start=1 << 40).reshape(count, 4)
    out = []
    for k in range(count):
        n = BATCH_SIZES[min(int(draws[k, 0] * len(BATCH_SIZES)), len(BATCH_SIZES) - 1)]
        chi = 2.0 + draws[k, 1]
        mob = 10.0 ** (-4.0 + 2.0 * draws[k, 2])
        r = 0.05 + 0.10 * draws[k, 3]
        prm = base.replace(nx=n, ny=n, chi=chi, mobility=mob, precision=MIXED)
        geo = dataclasses.replace(geo0, radius=r, seed=seed + k)
        out.append((prm, geo))
    return out
