"""Temporally blocked multigrid passes (one launch per level and direction
for the FP32 5-point and 13-point hierarchies: the smoothing steps, the
residual and its restriction in shared memory) against the separate launches of the same
V-cycle (CAHN_MG_FUSED=0).  Each node is computed with the same operations,
so single solves, whole steps and batched steps agree bit for bit."""
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


# the single-block tail off in both (the fused default; the separate
# launches keep it unless told otherwise)
FUSED = {"CAHN_MG_FUSED": None, "CAHN_MG_TAIL": "0"}
SEPARATE = {"CAHN_MG_FUSED": "0", "CAHN_MG_TAIL": "0"}
# grids: square, ragged in both directions, odd tile counts, the large workload
GRIDS = {"64x64": (64, 64, 2.0), "40x22": (40, 22, 2.0), "96x130": (96, 130, 1.0),
         "160x70": (160, 70, 2.0), "1024x1024": (1024, 1024, 4.0)}


def _setup(nx, ny, lx, **kw):
    prm = inputs.config_small()[0].replace(nx=nx, ny=ny, lx=lx, precision=inputs.MIXED, **kw)
    prm = prm.replace(eps=max(prm.eps, 2 * prm.ly / prm.ny))
    geo = inputs.Protrusions(h_b=0.3, centres=(0.5 * prm.lx,), radius=0.2 * prm.ly,
                             noise=1e-3, seed=3)
    return prm, inputs.initial_state(prm, geo)


@pytest.mark.parametrize("tail", ["1", "0"])
@pytest.mark.parametrize("grid", list(GRIDS))
def test_fused_solves_bitwise(grid, tail):
    prm, state = _setup(*GRIDS[grid], rtol=1e-12, max_iters=4000)
    rhs = inputs.random_field(prm, seed=11)

    def run():
        sim = binding.Simulation([prm], [state])
        out = [sim.solve(0, s, rhs)
               for s in (binding.SYS_PHI, binding.SYS_U, binding.SYS_V, binding.SYS_P)]
        assert all(code == 0 for _, code, _ in out)
        res = [(x.cpu().numpy(), st["iters"]) for x, _, st in out]
        sim.close()
        return res

    a = _with_env(dict(FUSED, CAHN_MG_TAIL=tail), run)
    b = _with_env(dict(SEPARATE, CAHN_MG_TAIL=tail), run)
    for (xa, ia), (xb, ib) in zip(a, b):
        assert ia == ib
        assert np.array_equal(xa, xb)


@pytest.mark.parametrize("graph", [0, 1])
def test_fused_steps_bitwise(graph):
    """Five steps of the 1024^2 workload in mixed precision."""
    prm, geo, _ = inputs.config_large()
    prm = prm.replace(precision=inputs.MIXED, rtol=1e-10, use_graph=graph)
    state = inputs.initial_state(prm, geo)

    def run():
        sim = binding.Simulation([prm], [state])
        _, st = sim.step(5)
        out = sim.numpy(0)
        sim.close()
        return out, st[0]["iters"]

    a, ia = _with_env(FUSED, run)
    b, ib = _with_env(SEPARATE, run)
    assert ia == ib
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_fused_batch_bitwise():
    """A batch graph of four uneven instances."""
    cases = []
    for k, (n, m) in enumerate(((128, 128), (192, 96), (256, 256), (96, 130))):
        prm, state = _setup(n, m, 2.0, rtol=1e-10, use_graph=1)
        cases.append((prm.replace(chi=2.0 + 0.25 * k), state))

    def run():
        sim = binding.Simulation([c[0] for c in cases], [c[1] for c in cases])
        _, st = sim.step(3)
        out = [sim.numpy(k) for k in range(len(cases))]
        sim.close()
        return out, [s["iters"] for s in st]

    a, ia = _with_env(FUSED, run)
    b, ib = _with_env(SEPARATE, run)
    assert ia == ib
    for fa, fb in zip(a, b):
        for x, y in zip(fa, fb):
            assert np.array_equal(x, y)


def test_fused_cuts_launches():
    """The V-cycles of the 5-point hierarchies take one launch per level and
    direction: a 1024^2 mixed step launches far fewer kernels."""
    prm, geo, _ = inputs.config_large()
    prm = prm.replace(precision=inputs.MIXED, rtol=1e-10, use_graph=0)
    state = inputs.initial_state(prm, geo)

    def run():
        sim = binding.Simulation([prm], [state])
        sim.step(1)
        n = binding.cahn_last_launch_count(sim.ctx)
        sim.close()
        return n

    a = _with_env(FUSED, run)
    b = _with_env(SEPARATE, run)
    assert a < 0.75 * b, (a, b)


@pytest.mark.parametrize("fused", [None, "0"])
@pytest.mark.parametrize("grid", ["160x70", "1024x1024"])
def test_mg_down32_is_the_smoother_steps(grid, fused):
    """cahn_mg_down32's x is bit for bit three cahn_smooth32 steps from x = 0
    (the fused pass and the separate launches alike)."""
    import torch
    prm, state = _setup(*GRIDS[grid], rtol=1e-12)

    def run():
        sim = binding.Simulation([prm], [state])
        n = (prm.ny + 1, prm.nx)
        b = torch.as_tensor(inputs.random_field(prm, seed=5), device="cuda").float()
        b[0] = 0
        b[-1] = 0
        out = {}
        for sysid in (binding.SYS_U, binding.SYS_P):
            x = torch.full(n, float("nan"), device="cuda")
            binding.cahn_mg_down32(sim.ctx, 0, sysid, b.data_ptr(), x.data_ptr())
            y = [torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")]
            d = torch.zeros(n, device="cuda")
            cur = torch.zeros(n, device="cuda")
            for k in range(3):
                binding.cahn_smooth32(sim.ctx, 0, sysid, k, cur.data_ptr(), b.data_ptr(),
                                      d.data_ptr(), y[k % 2].data_ptr())
                cur = y[k % 2].clone()
            torch.cuda.synchronize()
            out[sysid] = (x.cpu().numpy(), cur.cpu().numpy())
        sim.close()
        return out

    res = _with_env({"CAHN_MG_FUSED": fused, "CAHN_MG_TAIL": None}, run)
    for sysid, (x, ref) in res.items():
        assert np.all(np.isfinite(x))
        assert np.array_equal(x, ref), (sysid, np.max(np.abs(x - ref)))
