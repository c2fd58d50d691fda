"""The paper's own parameter set (§5; the shear flow of §5.1; viscosity
ratio 4.3e5, Gamma2 = 1.25e6, Lambda = 1e-10) through the C ABI against the
FP64 oracle: ten steps at 64^2 (host loop and graph, FP64 and mixed) and
three at the paper's 256^2, per field.  Bars: 1e-10 (FP64), 1e-6 (mixed)."""
import numpy as np
import pytest

from oracle import cahn_oracle as O
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


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a)


@pytest.mark.parametrize("n,nsteps", [(64, 10), (256, 3)])
@pytest.mark.parametrize("precision,graph", [(inputs.FP64, 0), (inputs.FP64, 1),
                                             (inputs.MIXED, 1)])
def test_paper_parameter_set(n, nsteps, precision, graph):
    prm, geo, _ = inputs.config_paper(n)
    prm = prm.replace(precision=precision, use_graph=graph,
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
