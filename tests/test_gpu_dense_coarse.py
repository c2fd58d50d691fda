"""The exact dense coarsest-level solve of the constant-coefficient 5-point
hierarchies (x = P b, P the level's inverse or, for the singular pressure
operator, its wall-weighted pseudo-inverse) against the whole-spectrum
Chebyshev steps it replaces (CAHN_MG_DENSE=0).  Both make the V-cycle a
fixed linear preconditioner of the same system, so the solves agree to the
solver tolerance, and the exact coarse solve takes no more iterations."""
import os

import numpy as np
import pytest

from paper_1811_11842_gb300 import binding, inputs
from paper_1811_11842_gb300 import build as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    binding.load()


def _with_env(env, fn):
    old = {k: os.environ.get(k) for k in env}
    for k, v in env.items():
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = v
    try:
        return fn()
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a)


DENSE = {"CAHN_MG_DENSE": None}
CHEB = {"CAHN_MG_DENSE": "0"}
GRIDS = {"64x64": (64, 64, 2.0), "96x130": (96, 130, 1.0), "1024x1024": (1024, 1024, 4.0)}


def _setup(nx, ny, lx, **kw):
    prm = inputs.config_small()[0].replace(nx=nx, ny=ny, lx=lx, **kw)
    prm = prm.replace(eps=max(prm.eps, 2 * prm.ly / prm.ny))
    geo = inputs.Protrusions(h_b=0.3, centres=(0.5 * prm.lx,), radius=0.2 * prm.ly,
                             noise=1e-3, seed=3)
    return prm, inputs.initial_state(prm, geo)


@pytest.mark.parametrize("tail", ["0", "1"])
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("grid", list(GRIDS))
def test_pressure_solve_dense_against_chebyshev(grid, precision, tail):
    prec = inputs.MIXED if precision == "mixed" else inputs.FP64
    prm, state = _setup(*GRIDS[grid], precision=prec, rtol=1e-12, max_iters=4000)
    rhs = inputs.random_field(prm, seed=17)

    def run():
        sim = binding.Simulation([prm], [state])
        x, code, st = sim.solve(0, binding.SYS_P, rhs)
        sim.close()
        assert code == 0
        return x.cpu().numpy(), st["iters"][binding.SYS_P]

    env = {"CAHN_MG_TAIL": tail, "CAHN_MG_COOP": "0"}
    xd, idense = _with_env(dict(DENSE, **env), run)
    xc, icheb = _with_env(dict(CHEB, **env), run)
    assert idense <= icheb + 1, (idense, icheb)
    # the pressure is fixed up to a constant: compare the weighted-mean-free parts
    w = np.ones_like(xd)
    w[0] = w[-1] = 0.5
    xd = xd - (w * xd).sum() / w.sum()
    xc = xc - (w * xc).sum() / w.sum()
    assert rel(xd, xc) <= 1e-9


@pytest.mark.parametrize("graph", [0, 1])
def test_steps_dense_against_chebyshev(graph):
    """Three steps of the 1024^2 workload, mixed precision with FP64
    refinement to 1e-10: the fields agree far inside the mixed bar."""
    prm, geo, _ = inputs.config_large()
    prm = prm.replace(precision=inputs.MIXED, rtol=1e-10, use_graph=graph)
    state = inputs.initial_state(prm, geo)

    def run():
        sim = binding.Simulation([prm], [state])
        _, st = sim.step(3)
        out = sim.numpy(0)
        sim.close()
        return out, st[0]

    a, sa = _with_env(DENSE, run)
    b, sb = _with_env(CHEB, run)
    assert sa["status"] == 0 and sb["status"] == 0
    for name, x, y in zip(("phi", "u", "v", "p"), a, b):
        if name == "p":
            x = x - x.mean()
            y = y - y.mean()
        assert rel(x, y) <= 1e-8, name


def test_batch_instances_share_the_coarse_matrix():
    """Instances of equal grids share the host-side elimination; a batch
    of three (two equal) steps bit for bit as each instance alone."""
    prms, states = [], []
    for n, chi in ((128, 2.0), (128, 2.5), (192, 2.25)):
        prm, st = _setup(n, n, 2.0, precision=inputs.MIXED, rtol=1e-10, use_graph=1)
        prm = prm.replace(chi=chi)
        prms.append(prm)
        states.append(st)
    sim = binding.Simulation(prms, states)
    sim.step(2)
    for k in range(3):
        alone = binding.Simulation([prms[k]], [states[k]])
        alone.step(2)
        for x, y in zip(sim.numpy(k), alone.numpy(0)):
            assert np.array_equal(x, y), k
        alone.close()
    sim.close()
