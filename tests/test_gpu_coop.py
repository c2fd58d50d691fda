"""The cooperative V-cycle (the levels of an FP32 5-point hierarchy from a
given size down in one launch, passes separated by a grid barrier; the finer
levels as separate launches) against the separate launches
of the same V-cycle (CAHN_MG_COOP=0, CAHN_MG_TAIL=0): each node is computed
with the same operations, so single solves and whole steps agree bit for
bit; against the default multi-launch path (whose coarse levels run in the
single-block tail) they agree to rounding.  The cooperative form is opt-in
(CAHN_MG_COOP=1): on the 1024^2 workload its grid barriers cost more than
the kernel boundaries of a graph."""
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


SEPARATE = {"CAHN_MG_COOP": "0", "CAHN_MG_TAIL": "0"}
COOP = {"CAHN_MG_COOP": "1", "CAHN_MG_TAIL": "0", "CAHN_COOP_NODES": None}
# where the cooperative launch starts: the default level, every level, only
# the levels of at most 20,000 nodes (finer ones as separate launches)
COOP_FROM = {"default": None, "all": "1000000000", "coarse": "20000"}


def _setup(n, **kw):
    kw.setdefault("lx", 4.0 if n >= 1024 else 2.0)
    prm = inputs.config_small()[0].replace(nx=n, ny=n, precision=inputs.MIXED, **kw)
    prm = prm.replace(eps=max(prm.eps, 2 * prm.ly / prm.ny))
    geo = inputs.Protrusions(h_b=0.3, centres=(0.5 * prm.lx,), radius=0.2 * prm.ly,
                             noise=1e-3, seed=3)
    return prm, inputs.initial_state(prm, geo)


@pytest.mark.parametrize("start", list(COOP_FROM))
@pytest.mark.parametrize("n", [64, 160, 1024])
def test_coop_solves_bitwise(n, start):
    prm, state = _setup(n, rtol=1e-12, max_iters=4000)
    rhs = inputs.random_field(prm, seed=11)

    def run():
        sim = binding.Simulation([prm], [state])
        out = [sim.solve(0, s, rhs) for s in (binding.SYS_U, binding.SYS_V, binding.SYS_P)]
        assert all(code == 0 for _, code, _ in out)
        res = [(x.cpu().numpy(), st["iters"]) for x, _, st in out]
        sim.close()
        return res

    a = _with_env(dict(COOP, CAHN_COOP_NODES=COOP_FROM[start]), run)
    b = _with_env(SEPARATE, run)
    for (xa, ia), (xb, ib) in zip(a, b):
        assert ia == ib
        assert np.array_equal(xa, xb)


@pytest.mark.parametrize("graph", [0, 1])
def test_coop_steps_bitwise(graph):
    """Five steps of the 1024^2 workload, mixed precision (u and v V-cycles
    as two concurrent cooperative launches in graph mode)."""
    prm, geo, _ = inputs.config_large()
    prm = prm.replace(precision=inputs.MIXED, rtol=1e-10, use_graph=graph)
    state = inputs.initial_state(prm, geo)

    def run():
        sim = binding.Simulation([prm], [state])
        _, st = sim.step(5)
        out = sim.numpy(0)
        sim.close()
        return out, st[0]["iters"]

    a, ia = _with_env(COOP, run)
    b, ib = _with_env(SEPARATE, run)
    assert ia == ib
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_coop_matches_default_tail_path_to_rounding():
    prm, state = _setup(256, rtol=1e-12, max_iters=4000)
    rhs = inputs.random_field(prm, seed=12)

    def run():
        sim = binding.Simulation([prm], [state])
        x, code, st = sim.solve(0, binding.SYS_P, rhs)
        sim.close()
        assert code == 0
        return x.cpu().numpy(), st["iters"][binding.SYS_P]

    a, ia = _with_env({"CAHN_MG_COOP": "1", "CAHN_MG_TAIL": None}, run)
    b, ib = _with_env({"CAHN_MG_COOP": "0", "CAHN_MG_TAIL": None}, run)
    assert abs(ia - ib) <= 1
    assert rel(a, b) <= 1e-11


def test_coop_batch_bitwise():
    """A batch graph of three uneven instances, each V-cycle with its share
    of the device's cooperative capacity, against separate launches."""
    cases = []
    for k, n in enumerate((128, 192, 256)):
        prm, state = _setup(n, rtol=1e-10, use_graph=1)
        cases.append((prm.replace(chi=2.0 + 0.25 * k), state))

    def run():
        sim = binding.Simulation([c[0] for c in cases], [c[1] for c in cases])
        _, st = sim.step(3)
        out = [sim.numpy(k) for k in range(len(cases))]
        sim.close()
        return out, [s["iters"] for s in st]

    a, ia = _with_env(COOP, run)
    b, ib = _with_env(SEPARATE, run)
    assert ia == ib
    for fa, fb in zip(a, b):
        for x, y in zip(fa, fb):
            assert np.array_equal(x, y)
