"""The fully implicit variable-viscosity momentum (CAHN_MOM_IMPLICIT: the
whole stress div(2 eta D(v)) of Eq. 4.1 by Crank-Nicolson, u and v coupled,
CAHN_SYS_UV) through the C ABI against the FP64 oracle: the coupled
operator elementwise (FP64, FP32), single coupled solves, and whole steps
(host loop and graph, FP64 and mixed precision).  Bars: 1e-13 x max|A x|
for applies, 1e-10 per field for FP64 solves and steps, 1e-6 mixed."""
import numpy as np
import pytest

from oracle import cahn_oracle as O
from paper_1811_11842_gb300 import binding, inputs
from paper_1811_11842_gb300 import build as B

pytestmark = pytest.mark.gpu

GRIDS = {
    "64x64": dict(nx=64, ny=64, lx=2.0, ly=1.0),
    "40x22": dict(nx=40, ny=22, lx=2.0, ly=1.0),
    "160x70": dict(nx=160, ny=70, lx=2.0, ly=1.0),
}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    binding.load()


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a)


def _setup(grid, **kw):
    prm = inputs.config_small()[0].replace(momentum=inputs.MOMENTUM_IMPLICIT, **GRIDS[grid])
    prm = prm.replace(eps=max(prm.eps, 2 * prm.ly / prm.ny), **kw)
    geo = inputs.Protrusions(h_b=0.3, centres=(0.5 * prm.lx,), radius=0.2 * prm.ly,
                             noise=1e-3, seed=3)
    return prm, inputs.initial_state(prm, geo)


def _stack(a, b):
    return np.concatenate([a, b], axis=0)


@pytest.mark.parametrize("grid", list(GRIDS))
def test_coupled_apply_parity(grid):
    import torch
    prm, state = _setup(grid, precision=inputs.MIXED, flow_mode=inputs.FLOW_SHEAR, u_max=0.2)
    g = O.grid_of(prm)
    eta = O.viscosity(prm, state[0])
    xu, xv = inputs.random_field(prm, seed=9), inputs.random_field(prm, seed=10)
    ru, rv = O.visc_apply(prm, g, eta, xu, xv)
    ref = _stack(ru, rv)
    sim = binding.Simulation([prm], [state])
    y = sim.apply(0, binding.SYS_UV, _stack(xu, xv)).cpu().numpy()
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(y - ref)) <= 1e-13 * scale, np.max(np.abs(y - ref)) / scale
    x32 = torch.as_tensor(_stack(xu, xv), dtype=torch.float32, device="cuda").contiguous()
    y32 = torch.empty_like(x32)
    binding.cahn_apply32(sim.ctx, 0, binding.SYS_UV, x32.data_ptr(), y32.data_ptr())
    torch.cuda.synchronize()
    sim.close()
    assert np.max(np.abs(y32.cpu().numpy() - ref)) <= 2e-6 * scale


@pytest.mark.parametrize("precision", [inputs.FP64, inputs.MIXED])
@pytest.mark.parametrize("grid", list(GRIDS))
def test_coupled_solve_parity(grid, precision):
    prm, state = _setup(grid, precision=precision, rtol=1e-13, max_iters=20000,
                        flow_mode=inputs.FLOW_SHEAR, u_max=0.2)
    g = O.grid_of(prm)
    eta = O.viscosity(prm, state[0])
    bu, bv = inputs.random_field(prm, seed=11), inputs.random_field(prm, seed=12)
    ru, rv = O.visc_solve(prm, g, eta, bu, bv)
    sim = binding.Simulation([prm], [state])
    x, code, st = sim.solve(0, binding.SYS_UV, _stack(bu, bv))
    sim.close()
    assert code == 0, st
    assert rel(x.cpu().numpy(), _stack(ru, rv)) <= 1e-10, (st, rel(x.cpu().numpy(), _stack(ru, rv)))


@pytest.mark.parametrize("precision,graph", [(inputs.FP64, 0), (inputs.FP64, 1),
                                             (inputs.MIXED, 0), (inputs.MIXED, 1)])
def test_implicit_momentum_steps(precision, graph):
    """20 steps of the 64^2 workload with the implicit momentum, per field."""
    prm, geo, nsteps = inputs.config_small()
    prm = prm.replace(momentum=inputs.MOMENTUM_IMPLICIT, precision=precision, use_graph=graph,
                      rtol=1e-10 if precision == inputs.MIXED else 1e-12)
    state = inputs.initial_state(prm, geo)
    sim = binding.Simulation([prm], [state])
    _, st = sim.step(nsteps)
    got = sim.numpy(0)
    sim.close()
    ref = O.run(prm.replace(precision=inputs.FP64), *state, nsteps)
    tol = 1e-6 if precision == inputs.MIXED else 1e-10
    for name, gv, r in zip(("phi", "u", "v", "p"), got, (ref.phi, ref.u, ref.v, ref.p)):
        assert rel(gv, r) <= tol, (name, rel(gv, r), st[0]["iters"])


def test_implicit_and_split_differ_only_by_the_stress_treatment():
    """Uniform phi and a divergence-free Couette profile: both momentum
    forms keep the exact steady state (u = u_max y / Ly, v = p = 0)."""
    for mom in (inputs.MOMENTUM_SPLIT, inputs.MOMENTUM_IMPLICIT):
        prm = inputs.Params(nx=32, ny=16, flow_mode=inputs.FLOW_SHEAR, u_max=0.3, dt=1e-3,
                            momentum=mom, rtol=1e-13)
        u0, v0, p0 = inputs.initial_velocity(prm)
        phi = 0.3 * np.ones_like(u0)
        sim = binding.Simulation([prm], [(phi, u0, v0, p0)])
        sim.step(3)
        got = sim.numpy(0)
        sim.close()
        assert np.max(np.abs(got[1] - u0)) < 1e-11, mom
        assert np.max(np.abs(got[2])) < 1e-11 and np.max(np.abs(got[3])) < 1e-11


def test_adjoint_rejects_implicit_momentum():
    import torch
    prm, state = _setup("64x64")
    sim = binding.Simulation([prm], [state])
    dev = [torch.as_tensor(a, device="cuda").contiguous() for a in state]
    out = torch.empty_like(dev[0])
    bar = torch.zeros_like(dev[0])
    code, _, _ = binding.cahn_vjp(sim.ctx, 0, *[t.data_ptr() for t in dev], 2, 1,
                                  bar.data_ptr(), out.data_ptr(), check=False)
    sim.close()
    assert code == binding.CAHN_ERR_ARG
