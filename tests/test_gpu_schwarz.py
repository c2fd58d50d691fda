"""The one-level domain-decomposition preconditioner (CAHN_PC_SCHWARZ: the
paper's planned preconditioner, §4.1 and §6) through the C ABI against the
FP64 oracle: single solves of every system and whole steps, FP64 and mixed,
on grids with full and ragged subdomains; it must cut the Jacobi iteration
counts; small grids are refused."""
import numpy as np
import pytest

from oracle import cahn_oracle as O
from paper_1811_11842_gb300 import binding, inputs
from paper_1811_11842_gb300 import build as B

pytestmark = pytest.mark.gpu

GRIDS = {
    "64x64": dict(nx=64, ny=64, lx=2.0, ly=1.0),
    "96x130": dict(nx=96, ny=130, lx=1.0, ly=1.0),
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


def _state(prm):
    geo = inputs.Protrusions(h_b=0.3, centres=(0.5 * prm.lx,), radius=0.2 * prm.ly,
                             noise=1e-3, seed=3)
    return inputs.initial_state(prm.replace(eps=max(prm.eps, 2 * prm.ly / prm.ny)), geo)


@pytest.mark.parametrize("precision", [inputs.FP64, inputs.MIXED])
@pytest.mark.parametrize("grid", list(GRIDS))
@pytest.mark.parametrize("system", ["phi", "u", "p"])
def test_schwarz_solve_parity(grid, system, precision):
    prm = inputs.config_small()[0].replace(rtol=1e-13, max_iters=20000, precond=inputs.PC_SCHWARZ,
                                          precision=precision, **GRIDS[grid])
    state = _state(prm)
    sim = binding.Simulation([prm], [state])
    rhs = inputs.random_field(prm, seed=11)
    sysid = {"phi": 0, "u": 1, "p": 3}[system]
    x, code, st = sim.solve(0, sysid, rhs)
    sim.close()
    assert code == 0, st
    ref = O.solve_system(prm, O.init_state(prm, *state), system, rhs)
    assert rel(x.cpu().numpy(), ref) <= 1e-10, (st, rel(x.cpu().numpy(), ref))


def test_schwarz_nutrient_solve_parity():
    prm = inputs.config_nutrient()[0].replace(rtol=1e-13, precond=inputs.PC_SCHWARZ, nx=96, ny=64,
                                             dt=1e-3)
    phi, u, v, p = _state(prm)
    c = 0.6 + 0.3 * inputs.random_field(prm, seed=21, lo=0.0, hi=1.0)
    sim = binding.Simulation([prm], [(phi, u, v, p, c)])
    rhs = inputs.random_field(prm, seed=12)
    x, code, st = sim.solve(0, binding.SYS_C, rhs)
    sim.close()
    assert code == 0, st
    ref = O.solve_system(prm, O.init_state(prm, phi, u, v, p, c), "c", rhs)
    assert rel(x.cpu().numpy(), ref) <= 1e-10


@pytest.mark.parametrize("precision,graph", [(inputs.FP64, 0), (inputs.MIXED, 1)])
def test_schwarz_steps(precision, graph):
    prm, geo, nsteps = inputs.config_small()
    prm = prm.replace(precond=inputs.PC_SCHWARZ, precision=precision, use_graph=graph,
                      rtol=1e-10 if precision == inputs.MIXED else 1e-12)
    state = inputs.initial_state(prm, geo)
    sim = binding.Simulation([prm], [state])
    _, st = sim.step(nsteps)
    got = sim.numpy(0)
    sim.close()
    ref = O.run(prm.replace(precision=inputs.FP64), *state, nsteps)
    tol = 1e-6 if precision == inputs.MIXED else 1e-10
    for name, g, r in zip(("phi", "u", "v", "p"), got, (ref.phi, ref.u, ref.v, ref.p)):
        assert rel(g, r) <= tol, (name, rel(g, r), st[0]["iters"])


def test_schwarz_cuts_jacobi_iterations():
    """256^2: fewer iterations than point Jacobi for every system, a fraction
    of them for the stiff CG systems (measured: A_phi 10 -> 8, H 74 -> 28,
    L_h 1087 -> 293); the V-cycle's are lower still (6, 7, 8)."""
    prm = inputs.config_medium()[0].replace(rtol=1e-10, max_iters=20000)
    state = _state(prm)
    rhs = inputs.random_field(prm, seed=13)
    its = {}
    for name, pc in (("jacobi", inputs.PC_JACOBI), ("schwarz", inputs.PC_SCHWARZ),
                     ("mg", inputs.PC_MG)):
        sim = binding.Simulation([prm.replace(precond=pc)], [state])
        its[name] = [sim.solve(0, s, rhs)[2]["iters"][s] for s in (0, 1, 3)]
        sim.close()
    for k in range(3):
        assert its["schwarz"][k] < its["jacobi"][k], its
        assert its["mg"][k] <= its["schwarz"][k], its
    for k in (1, 2):
        assert its["schwarz"][k] < 0.5 * its["jacobi"][k], its


def test_schwarz_refuses_small_grids():
    prm = inputs.config_small()[0].replace(nx=40, ny=22, precond=inputs.PC_SCHWARZ)
    with pytest.raises(binding.CahnError) as e:
        binding.Simulation([prm], [_state(prm)])
    assert e.value.code == binding.CAHN_ERR_ARG
